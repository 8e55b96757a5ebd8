// 32-bit word kernels for N = 2^13 .. 2^17: a column pass of p1 = floor(n/2)
// stages, then a row pass of the rest (the same split as the 64-bit kernels).
#include "launch.cuh"

namespace ntt {

cudaError_t launch_w32_two(const PassLaunch<u32>& c, bool fwd)
{
    switch (c.n) {
    case 13: return launch_two_pass_w32<6, 7, 5, KMAX_ALL>(c, fwd);
    case 14: return launch_two_pass_w32<7, 7, 5, KMAX_ALL>(c, fwd);
    case 15: return launch_two_pass_w32<7, 8, 4, KMAX_ALL>(c, fwd);
    case 16: return launch_two_pass_w32<8, 8, 4, KMAX_ALL>(c, fwd);
    case 17: return launch_two_pass_w32<8, 9, 3, KMAX_ALL>(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
