// N = 2^13, geometry 2 (the other pass split): 7 column stages, then 6 row
// stages in tiles of 64 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(13, 2).p1 == 7 && geometry_of(13, 2).logc_r == 6, "geometry table");

cudaError_t launch_n13_g2(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 6, 6, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n13_g2(const JobsCtx& c, bool fwd) { return launch_jobs<7, 6, 6, KMAX_ALL>(c, fwd); }

}  // namespace ntt
