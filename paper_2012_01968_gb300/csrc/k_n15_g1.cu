// N = 2^15, geometry 1 (half the row tile): 7 column stages, then 8 row
// stages in tiles of 8 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(15, 1).p1 == 7 && geometry_of(15, 1).logc_r == 3, "geometry table");

cudaError_t launch_n15_g1(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 8, 3, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n15_g1(const JobsCtx& c, bool fwd) { return launch_jobs<7, 8, 3, KMAX_ALL>(c, fwd); }

}  // namespace ntt
