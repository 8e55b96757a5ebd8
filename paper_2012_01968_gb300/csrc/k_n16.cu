// Two-pass kernels for N = 2^16: 8 column stages, then 8 row stages.
#include "launch.cuh"

namespace ntt {

cudaError_t launch_n16(const LaunchCtx& c, bool fwd) { return launch_two_pass<8, 8, 4, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n16(const JobsCtx& c, bool fwd) { return launch_jobs<8, 8, 4, KMAX_ALL>(c, fwd); }

}  // namespace ntt
