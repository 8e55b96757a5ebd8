// Single-pass kernels, N = 2^1 .. 2^12 (one CTA holds a whole limb).
#include "launch.cuh"

namespace ntt {

cudaError_t launch_single(const LaunchCtx& c, bool fwd)
{
    switch (c.n) {
    case 1: return launch_single_n<1>(c, fwd);
    case 2: return launch_single_n<2>(c, fwd);
    case 3: return launch_single_n<3>(c, fwd);
    case 4: return launch_single_n<4>(c, fwd);
    case 5: return launch_single_n<5>(c, fwd);
    case 6: return launch_single_n<6>(c, fwd);
    case 7: return launch_single_n<7>(c, fwd);
    case 8: return launch_single_n<8>(c, fwd);
    case 9: return launch_single_n<9>(c, fwd);
    case 10: return launch_single_n<10>(c, fwd);
    case 11: return launch_single_n<11>(c, fwd);
    case 12: return launch_single_n<12>(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
