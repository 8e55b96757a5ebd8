// Two-pass kernels for N = 2^13: 6 column stages, then 7 row stages.
// Geometry 0 here; the autotuner's alternatives in k_n13_g1.cu and k_n13_g2.cu.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(13, 0).p1 == 6 && geometry_of(13, 0).logc_r == 5, "geometry table");

cudaError_t launch_n13_g1(const LaunchCtx& c, bool fwd);
cudaError_t launch_n13_g2(const LaunchCtx& c, bool fwd);
cudaError_t launch_jobs_n13_g1(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n13_g2(const JobsCtx& c, bool fwd);

cudaError_t launch_n13(const LaunchCtx& c, bool fwd)
{
    switch (c.geom) {
    case 0: return launch_two_pass<6, 7, 5, KMAX_ALL>(c, fwd);
    case 1: return launch_n13_g1(c, fwd);
    case 2: return launch_n13_g2(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_jobs_n13(const JobsCtx& c, bool fwd)
{
    switch (c.geom) {
    case 0: return launch_jobs<6, 7, 5, KMAX_ALL>(c, fwd);
    case 1: return launch_jobs_n13_g1(c, fwd);
    case 2: return launch_jobs_n13_g2(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
