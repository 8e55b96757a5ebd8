/*
 * ntt_gb300.h -- C ABI of the GB300 (sm_103a) negacyclic RNS NTT library.
 *
 * The library computes the forward and inverse negacyclic Number Theoretic
 * Transform of RNS polynomials (Kim, Jung, Park, Ahn, "Accelerating Number
 * Theoretic Transformations for Bootstrappable Homomorphic Encryption on
 * GPUs"):
 *
 *   forward (Sec. III-A merged form; output order of Algorithm 1):
 *     out[i] = sum_{n<N} a[n] * psi^{n (2 brv(i) + 1)}  mod q
 *   inverse (Sec. III-A, Psi^{-1} merged into the iNTT):
 *     a[n]   = N^{-1} * sum_{i<N} out[i] * psi^{-n (2 brv(i) + 1)}  mod q
 *
 * where brv is the log2(N)-bit reversal (forward outputs are in bit-reversed
 * order, as Algorithm 1 produces them; the inverse takes that order back to
 * natural order), q is an RNS prime with q = 1 mod 2N (Sec. III-B), and psi =
 * g^{(q-1)/2N} with g the smallest generator of Z_q^*.
 *
 * Data layout: a batch of polynomials is one device array of uint64_t words,
 * laid out [batch][L][N] (limb-contiguous: limb l of polynomial b starts at
 * word (b * L + l) * N).  Coefficients are residues in [0, q_l); results are
 * residues in [0, q_l).  Inputs outside [0, q_l) give unspecified results.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Device calls are asynchronous and stream-ordered; argument
 * errors are returned synchronously before anything is enqueued.  All calls
 * must run with the plan's device current.
 *
 * Concurrency: a plan owns one device work area (dependency counters of the
 * one-launch two-pass kernel, for N >= 2^13) and one host staging buffer.
 * Transform calls on one plan must therefore be ordered: issue them on one
 * stream, or order the streams with events.  Two plans are independent.  The
 * work area is sized at plan creation for batch 16; a call with a larger
 * batch * L grows it (a device synchronisation and an allocation), so make
 * one call at the largest batch before capturing calls into a CUDA graph.
 *
 * Errors: every call returns an ntt_status; NTT_OK is 0.  On error nothing is
 * enqueued and output arguments are left untouched.
 */
#ifndef NTT_GB300_H
#define NTT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ntt_status {
    NTT_OK = 0,
    NTT_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad option */
    NTT_ERR_BAD_PRIME = 2,    /* composite, q != 1 mod 2N, or q outside (2^32, 2^60) (32-bit plans: q >= 2^28) */
    NTT_ERR_MISALIGNED = 3,   /* a device pointer is not 16-byte aligned */
    NTT_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    NTT_ERR_OOM = 5,          /* device or host allocation failed */
    NTT_ERR_BUSY = 6,         /* admission refused (serving) */
    NTT_ERR_TIMEOUT = 7,      /* a bounded wait expired */
    NTT_ERR_DEVICE = 8,       /* a kernel reported an error status */
    NTT_ERR_LIMIT = 9         /* batch * levels above NTT_NOALLOC_MAX_LIMBS */
} ntt_status;

/* Opaque plan: N, the primes, psi per prime and the device tables. */
typedef struct ntt_plan ntt_plan;

/* Twiddle supply (Sec. VII): precomputed table Psi with Shoup companions, or
 * on-the-fly twiddling (OT), which rebuilds the twiddles of the last stages
 * from two small per-prime factor tables with one extra Shoup product each.
 * A table plan holds N entries (16 B each) per prime; with PER_PASS its row
 * pass stages the twiddles of all but its last stage in shared memory and
 * reads the last stage's from the table in device memory (half of the table
 * per forward or inverse call), where OT on one stage keeps N/2 entries
 * and forms the last stage's twiddles from its factor tables. */
enum {
    NTT_TWIDDLE_AUTO = 0,
    NTT_TWIDDLE_TABLE = 1,
    NTT_TWIDDLE_OT = 2
};

/* Kernel organisation: for two-pass sizes (N >= 2^13) one persistent launch
 * that runs both passes with per-limb dependency counters (FUSED, the
 * default), or one launch per pass (PER_PASS); for every size, RADIX2 is the
 * paper's starting point (Sec. VI): one launch per radix-2 stage with its
 * operands in global memory, and HIGH_RADIX its register-based high-radix
 * step (Sec. VI-B): one launch per radix_log2 stages, each thread running
 * them on 2^radix_log2 operands in registers.  Both with table twiddles only,
 * kept for comparison.  Results are identical. */
enum {
    NTT_KERNEL_AUTO = 0,
    NTT_KERNEL_FUSED = 1,
    NTT_KERNEL_PER_PASS = 2,
    NTT_KERNEL_RADIX2 = 3,
    NTT_KERNEL_HIGH_RADIX = 4,
    NTT_KERNEL_CLUSTER = 5
};
/* NTT_KERNEL_CLUSTER (N = 2^10 .. 2^12, table twiddles): each limb on a
 * thread-block cluster of N / 512 CTAs on as many SMs, two passes (floor(n/2)
 * column stages, then the rest, Sec. VI-C's decomposition) with the
 * transposition between them through distributed shared memory: one global
 * read and one write per limb per launch, for the latency of few-limb calls
 * (a one-pass CTA runs all n stages of its limb on one SM).  ntt_execute with
 * both operations runs forward and inverse in one launch.  The plan's table
 * is laid out for these passes.  Results are identical to the other
 * organisations. */

/* Pass geometries of the two-pass sizes (N >= 2^13, FUSED and PER_PASS):
 * the radix split N = 2^p1 x 2^(n-p1) and the height of the second pass's row
 * tiles (Sec. VI-C: the decomposition and the per-CTA tile are tuning
 * parameters).  0 is the default split p1 = floor(n/2); 1 halves the row tile;
 * 2 moves one stage to the other pass (ntt_plan_info reports the result). */
enum {
    NTT_GEOMETRY_DEFAULT = 0,
    NTT_GEOMETRY_SMALL_ROW_TILE = 1,
    NTT_GEOMETRY_ALT_SPLIT = 2
};

typedef struct ntt_plan_opts {
    uint32_t twiddle_mode;    /* NTT_TWIDDLE_*; AUTO: OT (ot_stages, default 1) for N >= 2^13, TABLE below */
    uint32_t ot_stages;       /* OT: final stages built on the fly, 1 or 2 (0 = 1) */
    uint32_t kernel;          /* NTT_KERNEL_* */
    uint32_t geometry;        /* NTT_GEOMETRY_*; must be 0 for N <= 2^12 and for RADIX2 */
    uint32_t flags;           /* NTT_PLAN_* bits */
    uint32_t radix_log2;      /* HIGH_RADIX: stages per launch, 1..5 (0 = 4, radix 16); else 0 */
    uint32_t ctas_per_sm;     /* FUSED two-pass sizes: persistent CTAs per SM of the plan's
                               * launches, 1..8, capped by what fits (0 = as many as fit, 2).
                               * 1 leaves room on every SM for a launch on another stream to
                               * run beside it; see NTT_CTAS_PER_SM_NOTE below */
    uint32_t reserved;        /* must be zero */
} ntt_plan_opts;

/* NTT_CTAS_PER_SM_NOTE: a fused launch ends in a tail where its last units
 * run on few SMs, and its passes meet at limb boundaries where units wait for
 * the previous pass of their limb.  With two persistent CTAs per SM (the
 * default) a launch on a second stream can start only as the first launch's
 * CTAs exit.  With one CTA per SM two launches on two streams run side by
 * side, each filling the other's waits: measured faster when two or more
 * streams issue transforms, slower for one stream alone. */

/* Keep the plan's twiddle table resident in L2 across calls: plan creation
 * raises this CUDA context's persisting-L2 limit (cudaLimitPersistingL2CacheSize,
 * a per-context runtime limit) to cover the table, up to the device maximum,
 * and the plan's own calls (ntt_forward / ntt_inverse and their variants) carry
 * an L2 access-policy window over it (hits persist, misses stream).  Batch and
 * server launches, which mix plans, do not. */
#define NTT_PLAN_L2_TWIDDLES 1u

/*
 * Create a plan for N-point transforms over the L primes primes[0..L-1].
 *   N      : power of two, 2 <= N <= 131072 (2^17).
 *   primes : host array of L primes, each with q = 1 mod 2N and
 *            2^32 < q < 2^60 (copied; the caller keeps ownership).
 *   L      : 1 <= L <= 4096.
 *   opts   : NULL for defaults.
 * The plan (host object, device tables of 16 * N * L bytes in table mode, and
 * the work area) belongs to the library until ntt_plan_destroy.  It is created on the
 * current CUDA device.  Errors: NTT_ERR_INVALID_ARG, NTT_ERR_BAD_PRIME,
 * NTT_ERR_OOM, NTT_ERR_CUDA; *out is left untouched on error.
 * (Paper: the precomputed tables of Sec. IV "Precomputed table size with
 * batching" and Sec. VII.)
 */
ntt_status ntt_plan_create(ntt_plan** out, uint32_t N, const uint64_t* primes, uint32_t L,
                           const ntt_plan_opts* opts);

/* Free a plan.  NULL is allowed.  Work that uses the plan must have finished. */
void ntt_plan_destroy(ntt_plan* plan);

/*
 * A second plan for the same transform that shares `plan`'s device tables
 * (twiddles, OT factors, prime constants: no new 16 N L bytes) but has its own
 * work area, status word and staging, so that calls on the two plans may
 * overlap in time (e.g. one plan per stream).  Sharing one table also keeps
 * it in L2 for both.  The tables are freed with the last plan that shares
 * them; the plans are destroyed independently.  Must run with the plan's
 * device current.  Errors: NTT_ERR_INVALID_ARG, NTT_ERR_OOM, NTT_ERR_CUDA.
 */
ntt_status ntt_plan_clone(ntt_plan** out, const ntt_plan* plan);

/*
 * Change the persistent CTAs per SM of the plan's fused launches (the
 * ctas_per_sm plan option, 0..8, 0 = as many as fit), e.g. on a clone that
 * runs alone on one stream while its source runs beside other streams.
 * Takes effect for calls made after it returns; do not call it while another
 * thread issues calls on the same plan.  Errors: NTT_ERR_INVALID_ARG (NULL,
 * ctas_per_sm > 8).
 */
ntt_status ntt_plan_set_ctas_per_sm(ntt_plan* plan, uint32_t ctas_per_sm);

/*
 * In-place forward transform of `batch` polynomials at device address `data`
 * (layout [batch][L][N], 16-byte aligned, caller-owned).  Input in natural
 * coefficient order, output in bit-reversed order (Algorithm 1).  All
 * batch * L limbs run in one launch (N <= 2^12, or the fused two-pass kernel)
 * or one launch per pass (PER_PASS) (batching, Sec. V / VI-A).
 * Errors: NTT_ERR_INVALID_ARG (NULL, batch == 0), NTT_ERR_MISALIGNED,
 * NTT_ERR_OOM (growing the plan's work area failed), NTT_ERR_CUDA (launch
 * failure).
 */
ntt_status ntt_forward(const ntt_plan* plan, uint64_t* data, uint32_t batch, void* stream);

/* In-place inverse transform (bit-reversed order in, natural order out,
 * N^{-1} applied).  Same arguments and errors as ntt_forward. */
ntt_status ntt_inverse(const ntt_plan* plan, uint64_t* data, uint32_t batch, void* stream);

/*
 * Level-aware variants: transform only the first `levels` primes of the plan
 * (1 <= levels <= L); data is laid out [batch][levels][N].  A polynomial at a
 * lower HE level carries fewer RNS limbs (Sec. III-B).
 */
ntt_status ntt_forward_levels(const ntt_plan* plan, uint64_t* data, uint32_t batch,
                              uint32_t levels, void* stream);
ntt_status ntt_inverse_levels(const ntt_plan* plan, uint64_t* data, uint32_t batch,
                              uint32_t levels, void* stream);

/*
 * c = a (*) b, the element-wise product mod q_l of two polynomials in the
 * transform domain (the middle step of the convolution theorem, Sec. III-A).
 * a, b, c: device arrays [batch][L][N], 16-byte aligned; c may alias a or b.
 */
ntt_status ntt_mul_pointwise(const ntt_plan* plan, const uint64_t* a, const uint64_t* b,
                             uint64_t* c, uint32_t batch, void* stream);

/*
 * Negacyclic product in coefficient form (Sec. III-A: NTT, element-wise
 * product, iNTT):  c = a * b mod (X^N + 1), limb by limb mod q_l, for
 * `batch` pairs of polynomials [batch][L][N].  Both forward transforms run in
 * one launch (fused plans), then the element-wise product into c, then the
 * inverse of c.  With a fused plan and c aliasing a or b, the product is not
 * a separate pass: the inverse's first pass multiplies each tile of c by the
 * other factor's transform before its stages.  The factor that c does not
 * alias is left holding its forward transform (natural input order in,
 * bit-reversed transform out, as ntt_forward), and so are both when c aliases
 * neither; a and b must not overlap.  Errors as ntt_forward, and
 * NTT_ERR_INVALID_ARG for overlapping a and b.
 */
ntt_status ntt_mul_negacyclic(const ntt_plan* plan, uint64_t* a, uint64_t* b, uint64_t* c, uint32_t batch,
                              void* stream);

/* Operation flags for ntt_execute and ntt_execute_host. */
enum {
    NTT_OP_FORWARD = 1,
    NTT_OP_INVERSE = 2          /* with NTT_OP_FORWARD: forward, then inverse */
};

/*
 * The operations in `ops` on `batch` polynomials at device address `data`
 * (as ntt_forward / ntt_inverse): NTT_OP_FORWARD, NTT_OP_INVERSE, or both
 * (the forward transform, then the inverse of its result).  With both and a
 * plan of the fused two-pass kernel (N >= 2^13), the two transforms run in one
 * launch: the forward's column pass, its row pass, the inverse's row pass and
 * its column pass of every limb in one persistent kernel, each pass of a limb
 * starting when the previous pass of that limb has been written back (no
 * launch boundary between the directions).  Results equal ntt_forward then
 * ntt_inverse; the forward's result is written to `data` and read back by the
 * inverse, as with two calls.  Other plans make one call per direction.
 * The chained launch needs a work area for three times the limbs; the plan's
 * grows on first use as for ntt_forward.  Errors as ntt_forward, and
 * NTT_ERR_INVALID_ARG for bad `ops`.
 */
ntt_status ntt_execute(const ntt_plan* plan, uint64_t* data, uint32_t batch, uint32_t ops, void* stream);

/*
 * Host-memory convenience call: copy `batch` polynomials from host_in to the
 * device, apply the operations in `ops` (forward, inverse, or forward then
 * inverse), copy the result to host_out, and wait for completion.  The data
 * moves in segments (limb ranges or groups of polynomials) over three internal
 * streams of the plan, so the copies of one segment overlap the transforms of
 * the others; the work starts after everything enqueued earlier on `stream`.
 * Uses a device staging buffer, the streams and per-stream work areas owned by
 * the plan (grown on first use and kept until ntt_plan_destroy); host_in and
 * host_out may be the same array and should be page-locked for full copy
 * bandwidth.  Calls on one plan are serialised.  Returns NTT_ERR_DEVICE when
 * the plan's status word is set after the call (a bounded wait of the kernels
 * ran out; see ntt_plan_device_status, which still reads and clears it).
 */
ntt_status ntt_execute_host(const ntt_plan* plan, const uint64_t* host_in, uint64_t* host_out,
                            uint32_t batch, uint32_t ops, void* stream);

/*
 * Asynchronous form of ntt_execute_host: enqueues the same copies and
 * transforms (in two segments) and returns without waiting; the work starts
 * after everything enqueued earlier on `stream`, and `stream` is ordered after
 * the last copy-out, so host_out holds the result once `stream` has reached
 * this point (e.g. after cudaStreamSynchronize(stream)).  host_in and
 * host_out must stay valid, and host_in unchanged, until then.  The plan has
 * two staging buffers, used by alternate calls: calls issued on two
 * alternating streams overlap (one call's copy-in runs while the previous
 * call is transformed and copied out), while calls on one stream follow one
 * another.  Errors as ntt_execute_host; on an error the plan's host streams
 * are drained before returning.
 */
ntt_status ntt_execute_host_async(const ntt_plan* plan, const uint64_t* host_in, uint64_t* host_out,
                                  uint32_t batch, uint32_t ops, void* stream);

/*
 * No-allocation transform.  The paper has no counterpart: this is a library
 * interface for callers that may not allocate device memory while they run,
 * e.g. a serving loop whose device memory is fully reserved up front, code
 * called back from inside a memory allocator, or a runtime that forbids
 * allocation in its steady state.  ntt_forward / ntt_inverse may grow the
 * plan's work area (a device synchronisation and an allocation) when a call
 * has more limbs than the plan was sized for; this call never allocates,
 * frees or synchronises.
 *
 * op is NTT_OP_FORWARD or NTT_OP_INVERSE (exactly one); data, batch and
 * levels (1 <= levels <= L, layout [batch][levels][N]) are as for
 * ntt_forward_levels / ntt_inverse_levels, and results are identical to
 * theirs.  The call's scratch (dependency counters of the one-launch two-pass
 * kernel, 4 + 2 * batch * levels words) lives in a fixed device array of this
 * library, one per device, sized for NTT_NOALLOC_MAX_LIMBS limbs (64 KB).  It
 * starts at zero when the library is loaded on a device, and every launch
 * leaves it at zero again.
 *
 * The first call on a device does a one-time set-up (it looks up the
 * array's device address, which may load the library's device code): make
 * it before any stream capture.  The address belongs to the CUDA context:
 * after cudaDeviceReset, or under a context the caller made current itself,
 * the next call looks it up again (and starts from a zeroed array), so that
 * first call in the new context also belongs before any capture.  All calls to this function on one device
 * share the one array, whatever the plan: calls that overlap in time (on
 * different streams, or from different host threads without ordering) race
 * on it and give wrong results.  Order them on one stream or with events.
 * Must run with the plan's device current.
 *
 * Errors: NTT_ERR_INVALID_ARG (NULL, batch or levels 0, levels > L, bad op,
 * current device is not the plan's), NTT_ERR_MISALIGNED, NTT_ERR_LIMIT
 * (batch * levels > NTT_NOALLOC_MAX_LIMBS; nothing is enqueued), NTT_ERR_CUDA
 * (set-up or launch failure).
 */
#define NTT_NOALLOC_MAX_LIMBS 8192u

ntt_status ntt_transform_noalloc(const ntt_plan* plan, uint64_t* data, uint32_t batch,
                                 uint32_t levels, uint32_t op, void* stream);

/*
 * Uneven batches (Sec. V and Sec. VI-A batch the limbs of equal transforms;
 * this extends it to jobs of different sizes, levels and directions, as met
 * at the different levels of an HE computation).
 *
 * A job transforms one array [batch][levels][N] of one plan in place, in one
 * direction.  ntt_batch_submit runs a list of jobs in few launches:
 *   - jobs of fused plans (N >= 2^13) with the default geometry go into one
 *     launch per OT setting and 128 jobs, whatever their sizes and directions (a
 *     persistent kernel in which each (size, direction) group runs its two
 *     passes and CTAs move to another group when theirs has no work left);
 *     with default plans a submission of any mix is one launch;
 *   - jobs of fused plans with another geometry share launches of one size,
 *     direction and OT setting, up to 16 jobs per launch;
 *   - jobs of N <= 2^12 or of other kernel organisations run one by one.
 * These launches run concurrently on the batch object's internal streams,
 * forked from and joined back to `stream`; the whole submission is ordered
 * on `stream` like a single call.  Results equal those of
 * ntt_forward_levels / ntt_inverse_levels on each job.  The mixed launch's job
 * descriptors (tensor maps and tables) are uploaded on `stream` when they
 * differ from the previous submission's, into the next of four descriptor
 * generations; a submission repeated on the same arrays (or replayed from a
 * captured graph) reuses the latest generation.  The host waits only when a
 * generation is reused while the submission that last used it is still
 * running (four submissions with different descriptors in flight): the call
 * does not drain `stream`.
 *
 * Ownership and concurrency: the caller keeps its plans and arrays alive until
 * the work has finished; arrays of one submission must not overlap (rejected).
 * The batch object owns internal streams, a work area and the descriptor
 * arrays; calls on one batch object must not overlap in time.  The work area
 * grows when a submission needs more (a device synchronisation and an
 * allocation), and a submission whose descriptors changed uploads them, which
 * a capture refuses; so make one eager submission of the same jobs before
 * capturing a submission into a CUDA graph.  The graph reads that
 * generation's descriptors: while it is in use, submit at most three other
 * sets of jobs on that batch object.  Must run with the batch's device
 * current.
 */
typedef struct ntt_batch ntt_batch;

typedef struct ntt_job {
    const ntt_plan* plan;
    uint64_t* data;           /* device, 16-byte aligned, [batch][levels][N] of the plan's N */
    uint32_t batch;           /* >= 1 */
    uint32_t levels;          /* 1 <= levels <= plan L: the plan's first `levels` primes */
    uint32_t op;              /* NTT_OP_FORWARD or NTT_OP_INVERSE */
    uint32_t reserved;        /* must be zero */
} ntt_job;

/* Create a batch object on the current device.  Errors: NTT_ERR_INVALID_ARG,
 * NTT_ERR_OOM, NTT_ERR_CUDA. */
ntt_status ntt_batch_create(ntt_batch** out);

/* Free a batch object.  NULL is allowed.  Work it enqueued must have finished. */
void ntt_batch_destroy(ntt_batch* batch);

/* Enqueue njobs jobs.  Errors (nothing is enqueued): NTT_ERR_INVALID_ARG
 * (NULL, njobs == 0, a bad job field, overlapping arrays, a plan or batch of
 * another device), NTT_ERR_MISALIGNED, NTT_ERR_OOM (growing the work area);
 * NTT_ERR_CUDA if a launch fails (earlier launches stay enqueued). */
ntt_status ntt_batch_submit(ntt_batch* batch, const ntt_job* jobs, uint32_t njobs, void* stream);

/* Device status word of the batch's fused launches (bits as for
 * ntt_plan_device_status).  Synchronises the device, reads and clears it. */
ntt_status ntt_batch_device_status(ntt_batch* batch, uint32_t* status);

/*
 * Serving: a request loop with admission by device memory and continuous
 * batching (a runtime around the transforms; the paper has no counterpart).
 *
 * A server owns a scheduler thread, `slots` streams with a batch object each,
 * and optionally a device arena for host-buffer requests.  Submitted
 * requests wait in a FIFO queue; the scheduler admits them from its head
 * while the bytes of all admitted requests stay within hbm_budget_bytes (and,
 * for NTT_REQ_HOST requests, the arena has room), and starts a batch (up to
 * max_batch_jobs requests) in the first free slot: copy-in of host requests,
 * one ntt_batch_submit, copy-out.  Requests arriving while batches are on the
 * device join the next free slot as memory frees up, so batches overlap.
 *
 * Request memory stays owned by the caller and must stay valid until the
 * request is done.  Device requests are transformed in place; host requests
 * are read from `data` and written to `host_out` (may be the same array;
 * page-locked for full copy bandwidth).  The server's plans and device must
 * stay current as for single calls; submit and wait may be called from any
 * host thread.
 */
#define NTT_REQ_HOST 1u           /* data / host_out are host memory */

typedef struct ntt_server ntt_server;

typedef struct ntt_server_opts {
    uint64_t hbm_budget_bytes;    /* bytes of admitted requests at any time (> 0) */
    uint64_t arena_bytes;         /* device staging for NTT_REQ_HOST requests (0: none) */
    uint32_t max_batch_jobs;      /* requests per batch (0: 64) */
    uint32_t slots;               /* batches in flight (0: 3; at most 16) */
    uint32_t max_queue;           /* waiting requests before NTT_ERR_BUSY (0: 2^20) */
    uint32_t reserved[3];         /* must be zero */
} ntt_server_opts;

typedef struct ntt_request {
    const ntt_plan* plan;
    uint64_t* data;               /* [batch][levels][N]: device array, or host input with NTT_REQ_HOST */
    uint64_t* host_out;           /* NTT_REQ_HOST: host output; otherwise ignored */
    uint32_t batch;
    uint32_t levels;              /* 1 <= levels <= plan L */
    uint32_t op;                  /* NTT_OP_FORWARD or NTT_OP_INVERSE */
    uint32_t flags;               /* 0 or NTT_REQ_HOST */
} ntt_request;

typedef struct ntt_request_times {
    int64_t submit_ns;            /* steady-clock times of submission, */
    int64_t start_ns;             /* of admission into a batch, */
    int64_t done_ns;              /* and of completion (0 while not done) */
    int64_t device_ns;            /* device time of the request's batch, from its
                                     first to its last operation (0 while not done) */
} ntt_request_times;

/* Create a server on the current device.  Errors: NTT_ERR_INVALID_ARG,
 * NTT_ERR_OOM, NTT_ERR_CUDA. */
ntt_status ntt_server_create(ntt_server** out, const ntt_server_opts* opts);

/* Drain: wait for every submitted request to finish, then free the server. */
void ntt_server_destroy(ntt_server* server);

/* Queue a request; *ticket identifies it.  Errors: NTT_ERR_INVALID_ARG (bad
 * field, or a request larger than the budget or the arena), NTT_ERR_MISALIGNED,
 * NTT_ERR_BUSY (max_queue requests already waiting: admission refused),
 * NTT_ERR_CUDA (a copy or launch of the server failed earlier; the server
 * takes no more requests). */
ntt_status ntt_server_submit(ntt_server* server, const ntt_request* request, uint64_t* ticket);

/* Wait up to timeout_ns for a request: its status (NTT_OK, or the error of
 * its batch: NTT_ERR_DEVICE when a bounded wait of the batch's kernels ran
 * out, its data then being invalid), or NTT_ERR_TIMEOUT if it is not done
 * yet. */
ntt_status ntt_server_wait(ntt_server* server, uint64_t ticket, uint64_t timeout_ns);

/* Timestamps of a request (for latency statistics). */
ntt_status ntt_server_request_times(ntt_server* server, uint64_t ticket, ntt_request_times* times);

/* Forget a finished request: its ticket, status and times are released (the
 * server otherwise keeps every request until ntt_server_destroy, so a
 * long-running loop should release each request once it has read what it
 * needs).  Errors: NTT_ERR_INVALID_ARG (unknown ticket), NTT_ERR_BUSY (the
 * request is not done yet; nothing is released). */
ntt_status ntt_server_release(ntt_server* server, uint64_t ticket);

/* Counters of the scheduler since the server was created, for diagnosing
 * latency: where a request's time went when its latency is far above the
 * batch's device time. */
typedef struct ntt_server_stats {
    uint64_t batches;             /* batches started */
    uint64_t requests;            /* requests finished */
    int64_t max_launch_ns;        /* longest host time to enqueue one batch (copies, launches, events) */
    int64_t max_loop_gap_ns;      /* longest interval between two passes of the scheduler loop */
    int64_t max_completion_gap_ns;/* longest interval, with a batch in flight, without a batch completing */
    int64_t max_device_ns;        /* longest device time of one batch */
    int64_t reserved[4];
} ntt_server_stats;

ntt_status ntt_server_stats_get(ntt_server* server, ntt_server_stats* stats);

/* One configuration tried by ntt_autotune, and its measured times. */
typedef struct ntt_tune_entry {
    ntt_plan_opts opts;       /* the configuration, as plan options */
    double forward_us;        /* mean device time of one ntt_forward call */
    double inverse_us;        /* mean device time of one ntt_inverse call */
    ntt_status status;        /* NTT_OK, or why the configuration was not timed */
    uint32_t reserved;
} ntt_tune_entry;

/*
 * Autotuner: the radix split and row tile (NTT_GEOMETRY_*), the kernel
 * organisation (FUSED, PER_PASS, RADIX2, HIGH_RADIX) and the twiddle supply (TABLE, OT of
 * the last 1 or 2 stages), the tuning parameters of Sec. VI-C and VII, are
 * picked by measurement on the current device.  Every compiled configuration
 * for N-point transforms of `batch` polynomials over primes[0..L-1] is timed:
 * `reps` calls (0: 20) of each direction after two warm-up calls, CUDA events
 * on an internal stream, inputs rotating over buffers that together exceed
 * twice the L2 (at most 1 GiB).  The fastest by forward + inverse time goes to
 * *best.
 *   entries / max_entries / count : optional; when entries is non-NULL, up to
 *     max_entries results are written in candidate order and *count (if
 *     non-NULL) receives the number of candidates.
 * The choice is cached per (device, N, L, batch, primes): a call with
 * entries == NULL returns the cached choice without timing when there is one
 * (then *count, if given, is 0).  A call with entries always times again and
 * refreshes the cache.  Allocates and frees device memory and plans, and
 * synchronises the device.  Errors: NTT_ERR_INVALID_ARG, NTT_ERR_BAD_PRIME,
 * NTT_ERR_OOM, NTT_ERR_CUDA; NTT_ERR_DEVICE when no configuration could be
 * timed.
 */
ntt_status ntt_autotune(uint32_t N, const uint64_t* primes, uint32_t L, uint32_t batch, uint32_t reps,
                        ntt_plan_opts* best, ntt_tune_entry* entries, uint32_t max_entries, uint32_t* count);

/*
 * 32-bit word transforms (Sec. IV, "32b vs. 64b word size": the same modulus
 * built from twice as many primes of half the width).  A separate plan type
 * over primes q < 2^28 with q = 1 mod 2N, residues held in uint32_t.  The
 * transform is the same negacyclic NTT as ntt_forward / ntt_inverse (same psi
 * rule: psi = g^{(q-1)/2N} for the smallest generator g of Z_q^*): for
 * N >= 2^13 the fused two-pass kernel (NTT_KERNEL_FUSED, the default) with
 * table twiddles or the last stage twiddled on the fly (OT), or one launch per
 * pass (NTT_KERNEL_PER_PASS, table); one pass below (table).
 */
typedef struct ntt_plan32 ntt_plan32;

/*
 * Create a 32-bit plan.  N as for ntt_plan_create; primes: host array of L
 * primes with q = 1 mod 2N and q < 2^28 (copied); 1 <= L <= 4096; kernel:
 * NTT_KERNEL_AUTO (= FUSED), NTT_KERNEL_FUSED or NTT_KERNEL_PER_PASS;
 * twiddle_mode: NTT_TWIDDLE_AUTO (OT of the last stage for fused two-pass
 * plans, table otherwise), NTT_TWIDDLE_TABLE or NTT_TWIDDLE_OT (fused two-pass
 * plans only).  Device tables of 8 * N * L bytes (table) or about half (OT)
 * and a work area, created on the current CUDA device.  Errors:
 * NTT_ERR_INVALID_ARG, NTT_ERR_BAD_PRIME, NTT_ERR_OOM, NTT_ERR_CUDA; *out is
 * left untouched on error.
 */
ntt_status ntt_plan32_create(ntt_plan32** out, uint32_t N, const uint32_t* primes, uint32_t L, uint32_t kernel,
                             uint32_t twiddle_mode);

/* Free a 32-bit plan.  NULL is allowed.  Work that uses it must have finished. */
void ntt_plan32_destroy(ntt_plan32* plan);

/*
 * In-place forward / inverse transform of `batch` polynomials of 32-bit
 * residues at device address `data` (layout [batch][L][N], 16-byte aligned,
 * caller-owned).  Orders and scaling as ntt_forward / ntt_inverse.  Errors:
 * NTT_ERR_INVALID_ARG (NULL, batch == 0, batch * L >= 2^32),
 * NTT_ERR_MISALIGNED, NTT_ERR_CUDA (launch failure).
 */
ntt_status ntt_forward32(const ntt_plan32* plan, uint32_t* data, uint32_t batch, void* stream);
ntt_status ntt_inverse32(const ntt_plan32* plan, uint32_t* data, uint32_t batch, void* stream);

/* psi for prime l (0 <= l < L) of a 32-bit plan, into *psi. */
ntt_status ntt_plan32_psi(const ntt_plan32* plan, uint32_t l, uint32_t* psi);

/* Device status word of a 32-bit plan, as ntt_plan_device_status. */
ntt_status ntt_plan32_device_status(const ntt_plan32* plan, uint32_t* status);

/*
 * Measurement helper for the roofline of the transform kernels (not part of
 * the transform path; the paper has no counterpart): times a register-only
 * loop of the forward butterfly (Shoup's lazy product, the range reduction
 * every other stage) on the current device and writes the butterflies per
 * second in units of 1e9.  Allocates and frees a small device buffer and
 * synchronises the device.  Errors: NTT_ERR_INVALID_ARG, NTT_ERR_CUDA.
 */
ntt_status ntt_measure_butterfly_rate(double* gbfly_per_s);

/* Plan facts, for callers and tests. */
typedef struct ntt_plan_info {
    uint32_t N, L;
    uint32_t log2_N;
    uint32_t passes;          /* kernel passes per transform (1 or 2) */
    uint32_t pass1_log2;      /* stages in the first pass */
    uint32_t twiddle_mode;    /* NTT_TWIDDLE_TABLE or NTT_TWIDDLE_OT */
    uint32_t ot_stages;       /* OT: final stages built on the fly */
    uint32_t device;          /* CUDA device ordinal */
    uint32_t kernel;          /* NTT_KERNEL_FUSED, _PER_PASS, _RADIX2 or _HIGH_RADIX */
    uint64_t device_bytes;    /* device memory held by the plan (tables) */
    uint32_t geometry;        /* NTT_GEOMETRY_* */
    uint32_t row_tile_log2;   /* rows per tile of the second pass (two-pass sizes), log2 */
    uint32_t radix_log2;      /* HIGH_RADIX: stages per launch; else 0 */
    uint32_t ctas_per_sm;     /* the option the plan was created with (0: as many as fit) */
} ntt_plan_info;

ntt_status ntt_plan_query(const ntt_plan* plan, ntt_plan_info* info);

/*
 * Device status word of the plan: bit 0 set when a bounded wait for a
 * dependency of the fused kernel ran out, bit 1 when a bounded wait for a
 * tile copy ran out (results of that call are then invalid).  Synchronises
 * the device, reads the word into *status and clears it.
 */
ntt_status ntt_plan_device_status(const ntt_plan* plan, uint32_t* status);

/* psi for prime l (0 <= l < L) of the plan, into *psi. */
ntt_status ntt_plan_psi(const ntt_plan* plan, uint32_t l, uint64_t* psi);

/* Static text for a status code (never NULL). */
const char* ntt_status_string(ntt_status status);

/* Text of the last CUDA error seen by this thread inside the library. */
const char* ntt_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NTT_GB300_H */
