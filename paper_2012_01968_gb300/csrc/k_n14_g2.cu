// N = 2^14, geometry 2 (the other pass split): 6 column stages, then 8 row
// stages in tiles of 16 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(14, 2).p1 == 6 && geometry_of(14, 2).logc_r == 4, "geometry table");

cudaError_t launch_n14_g2(const LaunchCtx& c, bool fwd) { return launch_two_pass<6, 8, 4, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n14_g2(const JobsCtx& c, bool fwd) { return launch_jobs<6, 8, 4, KMAX_ALL>(c, fwd); }

}  // namespace ntt
