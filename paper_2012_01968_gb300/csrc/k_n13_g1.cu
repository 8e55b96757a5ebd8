// N = 2^13, geometry 1 (half the row tile): 6 column stages, then 7 row
// stages in tiles of 16 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(13, 1).p1 == 6 && geometry_of(13, 1).logc_r == 4, "geometry table");

cudaError_t launch_n13_g1(const LaunchCtx& c, bool fwd) { return launch_two_pass<6, 7, 4, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n13_g1(const JobsCtx& c, bool fwd) { return launch_jobs<6, 7, 4, KMAX_ALL>(c, fwd); }

}  // namespace ntt
