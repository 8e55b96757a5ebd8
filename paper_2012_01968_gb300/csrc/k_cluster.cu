// Host side of the cluster kernel (ntt_cluster.cuh): N = 2^10 .. 2^12, one
// cluster of N / 512 CTAs per limb.
#include "launch.cuh"
#include "ntt_cluster.cuh"

namespace ntt {

namespace {

template <int NLOG, int MODE>
cudaError_t launch_cluster_mode(const LaunchCtx& c)
{
    using CF = ClusterCfg<NLOG>;
    auto kern = ntt_cluster_kernel<NLOG, MODE>;
    ClusterArgs a;
    a.data = c.data;
    a.primes = c.primes;
    a.tw = c.tw;
    a.L = c.L;
    a.limbs = c.limbs;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c.limbs * (unsigned)CF::CS, 1, 1);
    cfg.blockDim = dim3(CF::NT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CF::CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int NLOG>
cudaError_t launch_cluster_n(const LaunchCtx& c, bool fwd)
{
    if (c.chain) return launch_cluster_mode<NLOG, 2>(c);
    return fwd ? launch_cluster_mode<NLOG, 0>(c) : launch_cluster_mode<NLOG, 1>(c);
}

}  // namespace

cudaError_t launch_cluster(const LaunchCtx& c, bool fwd)
{
    // one cluster per limb: the grid's x extent is limbs x cluster size
    if ((u64)c.limbs * (1ull << (c.n - CLUSTER_TILE_LOG)) > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    switch (c.n) {
    case 10: return launch_cluster_n<10>(c, fwd);
    case 11: return launch_cluster_n<11>(c, fwd);
    case 12: return launch_cluster_n<12>(c, fwd);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntt
