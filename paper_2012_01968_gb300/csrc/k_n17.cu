// Two-pass kernels for N = 2^17: 8 column stages, then 9 row stages.
#include "launch.cuh"

namespace ntt {

cudaError_t launch_n17(const LaunchCtx& c, bool fwd) { return launch_two_pass<8, 9, 3, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n17(const JobsCtx& c, bool fwd) { return launch_jobs<8, 9, 3, KMAX_ALL>(c, fwd); }

}  // namespace ntt
