// The fused two-pass kernel on 32-bit words for N = 2^13 .. 2^17 (table
// twiddles, one job per launch): the pass split of the 64-bit kernels, column
// tiles of 32 words x 2^p1 rows and row tiles of 2^13 words (2^12 at 2^17).
#include "launch.cuh"

namespace ntt {

cudaError_t launch_w32_fused(const Fused32Launch& c, bool fwd)
{
    switch (c.n) {
    case 13: return launch_fused32<6, 7, 6, KMAX_ALL>(c, fwd);
    case 14: return launch_fused32<7, 7, 6, KMAX_ALL>(c, fwd);
    case 15: return launch_fused32<7, 8, 5, KMAX_ALL>(c, fwd);
    case 16: return launch_fused32<8, 8, 5, KMAX_ALL>(c, fwd);
    case 17: return launch_fused32<8, 9, 3, KMAX_ALL>(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
