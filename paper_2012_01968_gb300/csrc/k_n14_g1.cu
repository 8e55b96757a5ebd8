// N = 2^14, geometry 1 (half the row tile): 7 column stages, then 7 row
// stages in tiles of 16 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(14, 1).p1 == 7 && geometry_of(14, 1).logc_r == 4, "geometry table");

cudaError_t launch_n14_g1(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 7, 4, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n14_g1(const JobsCtx& c, bool fwd) { return launch_jobs<7, 7, 4, KMAX_ALL>(c, fwd); }

}  // namespace ntt
