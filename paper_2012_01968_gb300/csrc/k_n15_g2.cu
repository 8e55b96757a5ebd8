// N = 2^15, geometry 2 (the other pass split): 8 column stages, then 7 row
// stages in tiles of 32 rows.
#include "launch.cuh"

namespace ntt {

static_assert(geometry_of(15, 2).p1 == 8 && geometry_of(15, 2).logc_r == 5, "geometry table");

cudaError_t launch_n15_g2(const LaunchCtx& c, bool fwd) { return launch_two_pass<8, 7, 5, KMAX_ALL>(c, fwd); }
cudaError_t launch_jobs_n15_g2(const JobsCtx& c, bool fwd) { return launch_jobs<8, 7, 5, KMAX_ALL>(c, fwd); }

}  // namespace ntt
