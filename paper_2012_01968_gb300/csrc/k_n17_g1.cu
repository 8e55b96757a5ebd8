// N = 2^17, geometry 1 (half the row tile): 8 column stages, then 9 row
// stages in tiles of 4 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(17, 1).p1 == 8 && geometry_of(17, 1).logc_r == 2, "geometry table");

cudaError_t launch_n17_g1(const LaunchCtx& c, bool fwd) { return launch_two_pass<8, 9, 2, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n17_g1(const JobsCtx& c, bool fwd) { return launch_jobs<8, 9, 2, KMAX_ALL>(c, fwd); }

}  // namespace ntt
