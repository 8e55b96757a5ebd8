// Two-pass kernels for N = 2^13: 6 column stages, then 7 row stages.
#include "launch.cuh"

namespace ntt {

cudaError_t launch_n13(const LaunchCtx& c, bool fwd) { return launch_two_pass<6, 7, 5, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n13(const JobsCtx& c, bool fwd) { return launch_jobs<6, 7, 5, KMAX_ALL>(c, fwd); }

}  // namespace ntt
