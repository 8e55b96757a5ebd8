// N = 2^16, geometry 1 (half the row tile): 8 column stages, then 8 row
// stages in tiles of 8 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(16, 1).p1 == 8 && geometry_of(16, 1).logc_r == 3, "geometry table");

cudaError_t launch_n16_g1(const LaunchCtx& c, bool fwd) { return launch_two_pass<8, 8, 3, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n16_g1(const JobsCtx& c, bool fwd) { return launch_jobs<8, 8, 3, KMAX_ALL>(c, fwd); }

}  // namespace ntt
