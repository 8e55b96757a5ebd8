// Two-pass kernels for N = 2^14: 7 column stages, then 7 row stages.
#include "launch.cuh"

namespace ntt {

cudaError_t launch_n14(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 7, 5, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n14(const JobsCtx& c, bool fwd) { return launch_jobs<7, 7, 5, KMAX_ALL>(c, fwd); }

}  // namespace ntt
