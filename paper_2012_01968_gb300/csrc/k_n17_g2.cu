// N = 2^17, geometry 2 (the other pass split): 7 column stages, then 10 row
// stages in tiles of 4 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(17, 2).p1 == 7 && geometry_of(17, 2).logc_r == 2, "geometry table");

cudaError_t launch_n17_g2(const LaunchCtx& c, bool fwd) { return launch_two_pass<7, 10, 2, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n17_g2(const JobsCtx& c, bool fwd) { return launch_jobs<7, 10, 2, KMAX_ALL>(c, fwd); }

}  // namespace ntt
