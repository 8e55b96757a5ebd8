// 32-bit word kernels for N = 2^1 .. 2^12: one pass, one CTA per limb.
#include "launch.cuh"

namespace ntt {

cudaError_t launch_w32_single(const PassLaunch<u32>& c, bool fwd)
{
    switch (c.n) {
    case 1: return launch_single_w32<1>(c, fwd);
    case 2: return launch_single_w32<2>(c, fwd);
    case 3: return launch_single_w32<3>(c, fwd);
    case 4: return launch_single_w32<4>(c, fwd);
    case 5: return launch_single_w32<5>(c, fwd);
    case 6: return launch_single_w32<6>(c, fwd);
    case 7: return launch_single_w32<7>(c, fwd);
    case 8: return launch_single_w32<8>(c, fwd);
    case 9: return launch_single_w32<9>(c, fwd);
    case 10: return launch_single_w32<10>(c, fwd);
    case 11: return launch_single_w32<11>(c, fwd);
    case 12: return launch_single_w32<12>(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
