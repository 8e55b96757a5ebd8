// N = 2^16, geometry 2 (the other pass split): 7 column stages, then 9 row
// stages in tiles of 8 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(16, 2).p1 == 7 && geometry_of(16, 2).logc_r == 3, "geometry table");

cudaError_t launch_n16_g2(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 9, 3, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n16_g2(const JobsCtx& c, bool fwd) { return launch_jobs<7, 9, 3, KMAX_ALL>(c, fwd); }

}  // namespace ntt
