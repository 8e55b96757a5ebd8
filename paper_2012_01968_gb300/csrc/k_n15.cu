// Two-pass kernels for N = 2^15: 7 column stages, then 8 row stages.
#include "launch.cuh"

namespace ntt {

cudaError_t launch_n15(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 8, 4, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n15(const JobsCtx& c, bool fwd) { return launch_jobs<7, 8, 4, KMAX_ALL>(c, fwd); }

}  // namespace ntt
