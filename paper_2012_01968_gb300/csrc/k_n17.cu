// Two-pass kernels for N = 2^17: 8 column stages, then 9 row stages.
// Geometry 0 here; the autotuner's alternatives in k_n17_g1.cu and k_n17_g2.cu.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(17, 0).p1 == 8 && geometry_of(17, 0).logc_r == 3, "geometry table");

cudaError_t launch_n17_g1(const LaunchCtx& c, bool fwd);
cudaError_t launch_n17_g2(const LaunchCtx& c, bool fwd);
cudaError_t launch_jobs_n17_g1(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n17_g2(const JobsCtx& c, bool fwd);

cudaError_t launch_n17(const LaunchCtx& c, bool fwd)
{
    switch (c.geom) {
    case 0: return launch_two_pass<8, 9, 3, KMAX_ALL>(c, fwd);
    case 1: return launch_n17_g1(c, fwd);
    case 2: return launch_n17_g2(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_jobs_n17(const JobsCtx& c, bool fwd)
{
    switch (c.geom) {
    case 0: return launch_jobs<8, 9, 3, KMAX_ALL>(c, fwd);
    case 1: return launch_jobs_n17_g1(c, fwd);
    case 2: return launch_jobs_n17_g2(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
