// Two-pass kernels for N = 2^16: 8 column stages, then 8 row stages.
// Geometry 0 here; the autotuner's alternatives in k_n16_g1.cu and k_n16_g2.cu.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(16, 0).p1 == 8 && geometry_of(16, 0).logc_r == 4, "geometry table");

cudaError_t launch_n16_g1(const LaunchCtx& c, bool fwd);
cudaError_t launch_n16_g2(const LaunchCtx& c, bool fwd);
cudaError_t launch_jobs_n16_g1(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n16_g2(const JobsCtx& c, bool fwd);

cudaError_t launch_n16(const LaunchCtx& c, bool fwd)
{
    switch (c.geom) {
    case 0: return launch_two_pass<8, 8, 4, KMAX_ALL>(c, fwd);
    case 1: return launch_n16_g1(c, fwd);
    case 2: return launch_n16_g2(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_jobs_n16(const JobsCtx& c, bool fwd)
{
    switch (c.geom) {
    case 0: return launch_jobs<8, 8, 4, KMAX_ALL>(c, fwd);
    case 1: return launch_jobs_n16_g1(c, fwd);
    case 2: return launch_jobs_n16_g2(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
