// Internal plan object and kernel dispatch interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <vector>

#include "ntt_gb300.h"
#include "device_types.cuh"
#include "ntt_pass.cuh"

namespace ntt {

// Pass split for N = 2^n: one pass for n <= SINGLE_PASS_MAX, else two passes
// of p1 = n - ceil(n/2) and p2 = ceil(n/2) stages.
constexpr int SINGLE_PASS_MAX = 12;
inline int split_p1(int n) { return n <= SINGLE_PASS_MAX ? n : n - (n + 1) / 2; }

// Geometries of the two-pass sizes (13 <= n <= 17): the pass split p1 (stages
// of the first, column-like pass) and the row tile height 2^logc_r of the
// second pass.  Index 0 is the default (p1 = split_p1(n)); 1 halves the row
// tile; 2 moves one stage to the other pass.  Each is compiled (k_nXX.cu,
// k_nXX_g1.cu, k_nXX_g2.cu) and picked per plan, by hand or by the autotuner.
// Limits: a column tile is 16 columns x 2^p1 rows (one TMA box, 2^p1 <= 256),
// a row tile at most 4096 words.
constexpr int kGeometries = 3;
struct Geometry {
    int p1, logc_r;
};
constexpr Geometry kGeometryTable[5][kGeometries] = {
    {{6, 5}, {6, 4}, {7, 6}},    // n = 13
    {{7, 5}, {7, 4}, {6, 4}},    // n = 14
    {{7, 4}, {7, 3}, {8, 5}},    // n = 15
    {{8, 4}, {8, 3}, {7, 3}},    // n = 16
    {{8, 3}, {8, 2}, {7, 2}},    // n = 17
};
constexpr Geometry geometry_of(int n, int g) { return kGeometryTable[n - 13][g]; }

// Round geometry of the pass that holds stage s (per-thread radix 2^KMAX), used
// to lay out the twiddle table in the slot order the kernels read.
#ifndef NTT_KMAX
#define NTT_KMAX 4      // stages per thread per round (per-thread radix 2^NTT_KMAX)
#endif
constexpr int KMAX_ALL = NTT_KMAX;
// 32-bit words of the fused kernel's work area for `limbs` limbs of one
// transform: four counters, a published-tile count per limb and the
// publication order.  A forward + inverse launch over `limbs` limbs needs
// the area of chain_work_limbs(limbs) limbs (four phases: eight counters and
// three of each per-limb array).
constexpr size_t fused_work_words(size_t limbs) { return 4 + 2 * limbs; }
constexpr size_t chain_work_limbs(size_t limbs) { return 3 * limbs + 2; }

struct StageSlot {
    int sl, K0, k;
};
// two_pass: stages [0, p1) form one pass and [p1, n) another (else one pass
// of n stages); kmax: stages per thread per round of those passes.
inline StageSlot stage_slot_params(int n, int p1, int s, bool two_pass, int kmax)
{
    const int s0 = (!two_pass || s < p1) ? 0 : p1;
    const int P = !two_pass ? n : (s < p1 ? p1 : n - p1);
    const int sl = s - s0;
    const int nr = (P + kmax - 1) / kmax;
    int K0 = 0;
    for (int r = 0; r < nr; ++r) {
        const int sz = P / nr + (r < P % nr ? 1 : 0);
        if (sl < K0 + sz) return StageSlot{sl, K0, sl - K0};
        K0 += sz;
    }
    return StageSlot{sl, 0, sl};
}
// The layout of the plans' kernels: one pass up to 2^SINGLE_PASS_MAX, else
// two, with KMAX_ALL stages per round.
inline StageSlot stage_slot_params(int n, int p1, int s)
{
    return stage_slot_params(n, p1, s, n > SINGLE_PASS_MAX, KMAX_ALL);
}

// Everything a launch needs (device pointers are the plan's).
struct LaunchCtx {
    u64* data;
    u32 limbs;               // polynomials x primes covered by the launch
    u32 L;                   // primes per polynomial (limb l uses prime l % L)
    const PrimeDev* primes;
    const Tw* tw;
    u32 tw_len;
    const Tw* ota_f;
    const Tw* otb_f;
    const Tw* ota_i;
    const Tw* otb_i;
    u32 n;
    u32 p1;
    u32 ots;                 // OT stages (0 = table mode)
    u32 separate_passes;     // 1: one launch per pass instead of the fused kernel
    u32 radix2;              // 1: one launch per radix-2 stage (natural-order table)
    u32 high_radix;          // k > 0: one launch per k stages in registers (natural-order table)
    u32* status;             // persistent device status word of the plan
    u32* work;               // fused kernel's work area (zero between launches)
    u32 work_limbs;          // limbs the work area covers (fused_work_words(work_limbs) words)
    cudaStream_t stream;
    u32 max_polls;           // bound of the fused kernel's waits (0: the default)
    u32 geom;                // geometry index (two-pass sizes; see kGeometryTable)
    const void* l2_base;     // L2 access-policy window of the launches (l2_bytes 0: none)
    size_t l2_bytes;
    float l2_hit;            // fraction of the window that persists
    // inverse through the fused kernel only: the other factor of an
    // element-wise product that the first pass applies (see JobCtx::mulb)
    const u64* mulb = nullptr;
    // fused two-pass plans, with fwd: the forward and then the inverse
    // transform in one launch (work area of chain_work_limbs(limbs) limbs)
    u32 chain = 0;
    u32 ctas_per_sm = 0;     // fused kernel: persistent CTAs per SM (0: as many as fit)
    u32 cluster = 0;         // 1: the cluster kernel (N = 2^10 .. 2^12; its own table layout)
};

cudaError_t launch_transform(const LaunchCtx& c, bool fwd);
// One limb per thread-block cluster (ntt_cluster.cuh, k_cluster.cu); with
// c.chain, forward and then inverse in one launch.
cudaError_t launch_cluster(const LaunchCtx& c, bool fwd);
// Table layout and sizes of the cluster kernel: two passes of floor(n/2) and
// ceil(n/2) stages, 3 stages per thread per round.
constexpr int CLUSTER_TABLE_KMAX = 3;
constexpr int CLUSTER_N_MIN = 10, CLUSTER_N_MAX = 12;

// One job of a multi-job fused launch: an array [batch][L][N] and the tables
// of its plan.
struct JobCtx {
    u64* data;
    u32 limbs;               // batch x L
    u32 L;                   // primes per polynomial (local limb l uses prime l % L)
    const PrimeDev* primes;
    const Tw* tw;
    u32 tw_len;
    const Tw* ota_f;
    const Tw* otb_f;
    const Tw* ota_i;
    const Tw* otb_i;
    // inverse only: the other factor of an element-wise product, in the same
    // layout as data; the first pass multiplies by it before its stages
    const u64* mulb = nullptr;
};

// Jobs of one size N = 2^n and one OT setting in one launch of the fused
// two-pass kernel (13 <= n <= 17, 1 <= njobs <= FUSED_MAX_JOBS).
constexpr int FUSED_MAX_JOBS = 16;
struct JobsCtx {
    const JobCtx* jobs;
    u32 njobs;
    u32 n;
    u32 ots;
    u32* status;
    u32* work;               // zero, fused_work_words(work_limbs) words
    u32 work_limbs;          // >= the jobs' limbs
    cudaStream_t stream;
    u32 max_polls;           // bound of every wait (0: the default)
    u32 geom = 0;            // geometry index shared by the jobs
    const void* l2_base = nullptr;   // L2 access-policy window (l2_bytes 0: none)
    size_t l2_bytes = 0;
    float l2_hit = 0.f;
    u32 chain = 0;                   // one job: forward, then inverse, in one launch
    u32 ctas_per_sm = 0;             // persistent CTAs per SM (0: as many as fit)
};
cudaError_t launch_fused_jobs(const JobsCtx& c, bool fwd);

// Jobs of different sizes (2^13 .. 2^17, plans of geometry 0) and directions
// in one launch (ntt_mixed.cuh, k_mixed.cu), at most MIXED_MAX_JOBS jobs.
// build_mixed makes the launch on the host: its job descriptors (tensor maps,
// mixed_job_bytes() per job, which the kernel reads from device memory) and
// its parameter block.  launch_mixed launches it with the descriptors at
// d_jobs (uploaded by the caller, in stream order before the launch).  The
// work area holds mixed_work_words() zeroed words.  stall_polls > 0 (test
// hook): every group's first-phase queue starts taken, waits bounded by it.
struct MixJobIn {
    JobCtx job;
    u32 n;                   // log2 N
    u32 fwd;                 // 1: forward
};
struct MixJob;
constexpr u32 MIXED_MAX_JOBS = 128;
size_t mixed_job_bytes();
size_t mixed_work_words(const MixJobIn* jobs, u32 njobs);
struct MixBuilt {
    std::vector<unsigned char> desc;      // the jobs' descriptors, mixed_job_bytes() each
    std::vector<unsigned char> params;    // the launch's parameter block
    u64 units_total = 0;
    u32 ots = 0;
    size_t work_words = 0;
};
cudaError_t build_mixed(const MixJobIn* jobs, u32 njobs, u32 ots, MixBuilt* out);
cudaError_t launch_mixed(const MixBuilt& m, const MixJob* d_jobs, u32* work, size_t work_words, u32* status,
                         u32 stall_polls, cudaStream_t s);
cudaError_t launch_pointwise(const PrimeDev* primes, u32 L, u32 n, const u64* a, const u64* b,
                             u64* out, u32 limbs, cudaStream_t s);

// per-n launchers (one translation unit each, compiled in parallel)
cudaError_t launch_single(const LaunchCtx& c, bool fwd);
cudaError_t launch_radix2(const LaunchCtx& c, bool fwd);
cudaError_t launch_high_radix(const LaunchCtx& c, bool fwd);
cudaError_t launch_n13(const LaunchCtx& c, bool fwd);
cudaError_t launch_n14(const LaunchCtx& c, bool fwd);
cudaError_t launch_n15(const LaunchCtx& c, bool fwd);
cudaError_t launch_n16(const LaunchCtx& c, bool fwd);
cudaError_t launch_n17(const LaunchCtx& c, bool fwd);
cudaError_t launch_jobs_n13(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n14(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n15(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n16(const JobsCtx& c, bool fwd);
cudaError_t launch_jobs_n17(const JobsCtx& c, bool fwd);

}  // namespace ntt

// Device tables of a plan, shared by the plan and its clones (ntt_plan_clone)
// and freed with the last of them.
struct NttPlanTables {
    ntt::PrimeDev* primes = nullptr;
    ntt::Tw* tw = nullptr;
    ntt::Tw* ota_f = nullptr;
    ntt::Tw* otb_f = nullptr;
    ntt::Tw* ota_i = nullptr;
    ntt::Tw* otb_i = nullptr;
    ~NttPlanTables()
    {
        cudaFree(primes);
        cudaFree(tw);
        cudaFree(ota_f);
        cudaFree(otb_f);
        cudaFree(ota_i);
        cudaFree(otb_i);
    }
};

struct ntt_plan {
    uint32_t N = 0, n = 0, L = 0;
    uint32_t p1 = 0, passes = 0;
    uint32_t twiddle_mode = 0, ot_stages = 0;
    int device = 0;
    std::vector<uint64_t> primes, psis;
    ntt::PrimeDev* d_primes = nullptr;
    ntt::Tw* d_tw = nullptr;
    uint32_t tw_len = 0;
    ntt::Tw* d_ota_f = nullptr;
    ntt::Tw* d_otb_f = nullptr;
    ntt::Tw* d_ota_i = nullptr;
    ntt::Tw* d_otb_i = nullptr;
    uint64_t device_bytes = 0;
    std::shared_ptr<NttPlanTables> tables;   // owner of d_primes .. d_otb_i
    uint32_t kernel = 0;                  // NTT_KERNEL_*
    uint32_t geom = 0;                    // geometry index (two-pass sizes)
    uint32_t flags = 0;                   // NTT_PLAN_* bits
    uint32_t radix_log2 = 0;              // HIGH_RADIX: stages per launch
    uint32_t ctas_per_sm = 0;             // fused launches: persistent CTAs per SM (0: as many as fit)
    float l2_hit = 0.f;                   // persisting fraction of the twiddle window
    uint32_t* d_status = nullptr;         // device status word (kernel error bits)
    uint32_t* d_work = nullptr;           // fused kernel's work area: fused_work_words(work_limbs) words
    uint32_t work_limbs = 0;
    std::mutex work_mu;
    // staging for ntt_execute_host: device copies of the data, two buffers
    // used by alternate calls; a copy-in stream, a copy-out stream and
    // kHostCompute compute streams (with one work area each), ordered per
    // segment by events
    static constexpr int kHostCompute = 2;
    static constexpr int kHostBuffers = 2;
    static constexpr int kHostSegments = 6;       // segments of a synchronous call
    static constexpr int kHostSegmentsAsync = 2;  // of an asynchronous call (calls overlap instead)
    std::mutex stage_mu;
    uint64_t* d_stage = nullptr;          // kHostBuffers x stage_bytes
    size_t stage_bytes = 0;               // per buffer
    uint32_t h_next = 0;                  // buffer of the next call
    cudaStream_t h_in = nullptr, h_out = nullptr, h_comp[kHostCompute] = {};
    cudaEvent_t hfork = nullptr, h_loaded[kHostSegments] = {}, h_done[kHostSegments] = {};
    // copy-out of each segment of the latest call on each buffer, with its
    // staging range [first, first + count) in limbs: a later call's copy-in of
    // an overlapping range of the same buffer waits for it
    cudaEvent_t h_out_done[kHostBuffers][kHostSegments] = {}, h_join = nullptr;
    uint32_t h_prev_first[kHostBuffers][kHostSegments] = {}, h_prev_count[kHostBuffers][kHostSegments] = {};
    uint32_t h_prev_segs[kHostBuffers] = {};
    uint32_t* d_hwork = nullptr;
    uint32_t hwork_limbs = 0;             // per compute stream

    ntt::LaunchCtx ctx(uint64_t* data, uint32_t limbs, uint32_t Lused, cudaStream_t s) const
    {
        ntt::LaunchCtx c;
        c.data = reinterpret_cast<ntt::u64*>(data);
        c.limbs = limbs;
        c.L = Lused;
        c.primes = d_primes;
        c.tw = d_tw;
        c.tw_len = tw_len;
        c.ota_f = d_ota_f;
        c.otb_f = d_otb_f;
        c.ota_i = d_ota_i;
        c.otb_i = d_otb_i;
        c.n = n;
        c.p1 = p1;
        c.ots = twiddle_mode == NTT_TWIDDLE_OT ? ot_stages : 0;
        c.separate_passes = kernel == NTT_KERNEL_PER_PASS ? 1u : 0u;
        c.radix2 = kernel == NTT_KERNEL_RADIX2 ? 1u : 0u;
        c.high_radix = kernel == NTT_KERNEL_HIGH_RADIX ? radix_log2 : 0u;
        c.status = d_status;
        c.work = d_work;
        c.work_limbs = work_limbs;
        c.stream = s;
        c.max_polls = 0;
        c.geom = geom;
        c.ctas_per_sm = ctas_per_sm;
        c.cluster = kernel == NTT_KERNEL_CLUSTER ? 1u : 0u;
        const bool win = (flags & NTT_PLAN_L2_TWIDDLES) && l2_hit > 0.f;
        c.l2_base = win ? (const void*)d_tw : nullptr;
        c.l2_bytes = win ? (size_t)L * tw_len * sizeof(ntt::Tw) : 0;
        c.l2_hit = l2_hit;
        return c;
    }

    // The same, for an array whose limb l uses prime prime0 + (l % Lview): the
    // tables are viewed from prime prime0 on.
    ntt::LaunchCtx ctx_range(uint64_t* data, uint32_t limbs, uint32_t Lview, uint32_t prime0, cudaStream_t s) const
    {
        ntt::LaunchCtx c = ctx(data, limbs, Lview, s);
        const size_t R = passes == 2 ? (size_t)1 << (n - p1) : 0;           // OT A entries per prime
        const size_t B = passes == 2 ? (size_t)(n - p1) << p1 : 0;          // OT B entries per prime
        c.primes = d_primes + prime0;
        c.tw = d_tw + (size_t)prime0 * tw_len;
        c.ota_f = d_ota_f ? d_ota_f + prime0 * R : nullptr;
        c.ota_i = d_ota_i ? d_ota_i + prime0 * R : nullptr;
        c.otb_f = d_otb_f ? d_otb_f + prime0 * B : nullptr;
        c.otb_i = d_otb_i ? d_otb_i + prime0 * B : nullptr;
        return c;
    }
};
