// Host side of the mixed-size launch (ntt_mixed.cuh): groups, job
// descriptors, and the three instantiations (table, OT of one or
// two stages).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "launch.cuh"
#include "ntt_mixed.cuh"

namespace ntt {

namespace {

template <int OTS>
cudaError_t launch_mixed_ots(const MixParams& prm, cudaStream_t s, u32 units_total, u32* grid_out)
{
    using LY = MixLayout<KMAX_ALL, OTS>;
    auto kern = ntt_mixed_kernel<KMAX_ALL, OTS>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int occ = 0;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::SMEM);
        if (attr_err == cudaSuccess)
            attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, LY::THREADS, LY::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const u64 slots = (u64)device_sm_count() * (u64)occ;
    const u32 grid = (u32)std::min<u64>(units_total, slots);
    *grid_out = grid;
    kern<<<grid, LY::THREADS, LY::SMEM, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

size_t mixed_job_bytes() { return sizeof(MixJob); }

size_t mixed_work_words(const MixJobIn* jobs, u32 njobs)
{
    std::vector<u64> limbs(MIX_MAX_GROUPS, 0);
    for (u32 i = 0; i < njobs; ++i) limbs[(jobs[i].n - MIX_FIRST_N) * 2 + (jobs[i].fwd ? 1 : 0)] += jobs[i].job.limbs;
    size_t w = 1;
    for (u64 l : limbs)
        if (l) w += mix_group_words(l);
    return w;
}

cudaError_t build_mixed(const MixJobIn* jobs, u32 njobs, u32 ots, MixBuilt* out)
{
    if (!out || njobs == 0 || njobs > (u32)MIX_MAX_JOBS || ots > 2) return cudaErrorInvalidValue;
    // groups: one per (size class, direction), in that order
    std::vector<std::vector<u32>> members(MIX_MAX_GROUPS);
    for (u32 i = 0; i < njobs; ++i) {
        if (jobs[i].n < (u32)MIX_FIRST_N || jobs[i].n >= (u32)(MIX_FIRST_N + MIX_CLASSES)) return cudaErrorInvalidValue;
        members[(jobs[i].n - MIX_FIRST_N) * 2 + (jobs[i].fwd ? 1 : 0)].push_back(i);
    }
    MixParams a{};
    std::vector<MixJob> hj(njobs);
    u32 nj = 0, ctl = 0;
    u64 units_total = 0;
    for (u32 key = 0; key < (u32)MIX_MAX_GROUPS; ++key) {
        if (members[key].empty()) continue;
        MixGroup& g = a.group[a.ngroups];
        g.cls = key / 2;
        g.fwd = key & 1;
        g.job0 = nj;
        g.njobs = (u32)members[key].size();
        const Geometry geo = geometry_of((int)(MIX_FIRST_N + g.cls), 0);
        const int p1 = geo.p1, cr = 1 << geo.logc_r, n = MIX_FIRST_N + (int)g.cls;
        const int row_tile = cr << (n - p1);
        u64 limbs = 0;
        for (u32 i : members[key]) {
            const JobCtx& J = jobs[i].job;
            MixJob& m = hj[nj];
            MixJobInfo& info = a.info[nj++];
            std::memset(&m, 0, sizeof(m));
            cudaError_t e = encode_tile_maps(J.data, J.limbs, (u32)n, p1, row_tile, &m.mapC, &m.mapR);
            if (e != cudaSuccess) return e;
            info.primes = J.primes;
            info.tw = J.tw;
            info.ota = g.fwd ? J.ota_f : J.ota_i;
            info.otb = g.fwd ? J.otb_f : J.otb_i;
            info.tw_len = J.tw_len;
            info.L = J.L;
            info.limb0 = (u32)limbs;
            limbs += J.limbs;
        }
        if (limbs >= (1ull << 28)) return cudaErrorInvalidValue;
        g.limbs = (u32)limbs;
        g.ctl = ctl;
        ctl += (u32)mix_group_words(limbs);
        units_total += limbs * (((1ull << n) >> p1 >> 4) + ((1ull << p1) / cr));
        ++a.ngroups;
    }
    out->desc.resize(sizeof(MixJob) * njobs);
    std::memcpy(out->desc.data(), hj.data(), out->desc.size());
    out->params.resize(sizeof(MixParams));
    std::memcpy(out->params.data(), &a, sizeof(a));
    out->units_total = units_total;
    out->ots = ots;
    out->work_words = (size_t)ctl + 1;
    return cudaSuccess;
}

cudaError_t launch_mixed(const MixBuilt& m, const MixJob* d_jobs, u32* work, size_t work_words, u32* status,
                         u32 stall_polls, cudaStream_t s)
{
    if (m.params.size() != sizeof(MixParams) || !d_jobs || m.ots > 2) return cudaErrorInvalidValue;
    if (!work || work_words < m.work_words) return cudaErrorInvalidValue;
    MixParams a;
    std::memcpy(&a, m.params.data(), sizeof(a));
    if (stall_polls) {
        static const u32 taken = 0x40000000u;
        for (u32 g = 0; g < a.ngroups; ++g) {
            cudaError_t e = cudaMemcpyAsync(work + a.group[g].ctl, &taken, sizeof(taken), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return e;
        }
    }
    a.jobs = d_jobs;
    a.ctl = work;
    a.status = status;
    a.ctl_words = (u32)m.work_words;
    a.max_polls = stall_polls ? stall_polls : 1u << 22;
    u32 grid = 0;
    const u32 units = (u32)std::min<u64>(m.units_total, 0xFFFFFFFFull);
    switch (m.ots) {
    case 0: return launch_mixed_ots<0>(a, s, units, &grid);
    case 1: return launch_mixed_ots<1>(a, s, units, &grid);
    default: return launch_mixed_ots<2>(a, s, units, &grid);
    }
}

}  // namespace ntt
