/*
 * CPU ORACLE for the negacyclic RNS NTT -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  The CUDA library never links, includes or
 * calls it, and this file uses nothing from the CUDA library.
 *
 * Everything here is plain and slow on purpose: every modular product is
 * ((unsigned __int128)a * b) % q, every sum and difference is reduced at once,
 * and each function follows the definition or algorithm it cites.
 *
 * Notation (paper: Kim, Jung, Park, Ahn, "Accelerating Number Theoretic
 * Transformations for Bootstrappable Homomorphic Encryption on GPUs"):
 *   N = 2^n, prime q with q = 1 mod 2N (Sec. III-B; Algorithm 1 input),
 *   psi = a primitive 2N-th root of unity mod q (psi_{2N,p} in Sec. III-A),
 *   brv(i) = the n-bit reversal of i (the "bit-reverse order" of Algorithm 1).
 *
 * Forward transform (Sec. III-A, merged form A_k = sum_n a_n psi^{n(2k+1)}),
 * with the output in the bit-reversed order that Algorithm 1 produces:
 *   out[i] = sum_{n<N} a[n] * psi^{n(2 brv(i) + 1)}  mod q.
 * Inverse transform: the map that undoes it (Sec. III-A: the Psi^{-1} twist
 * is merged into the iNTT):
 *   a[n] = N^{-1} * sum_{i<N} out[i] * psi^{-n(2 brv(i) + 1)}  mod q.
 * Negacyclic product (Sec. III-A):
 *   c_k = sum_{i<=k} a_i b_{k-i} - sum_{i>k} a_i b_{N+k-i}  mod q.
 *
 * Choice of psi (the paper only asks for a primitive 2N-th root): g is the
 * smallest integer >= 2 that generates Z_q^*, and psi = g^{(q-1)/2N} mod q.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* modular arithmetic on canonical residues                           */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - b) % q); }

u64 orc_powmod(u64 base, u64 e, u64 q)
{
    u64 r = 1 % q;
    base %= q;
    while (e) {
        if (e & 1) r = mulmod(r, base, q);
        base = mulmod(base, base, q);
        e >>= 1;
    }
    return r;
}

/* inverse by Fermat's little theorem (q prime, a != 0 mod q) */
u64 orc_invmod(u64 a, u64 q) { return orc_powmod(a, q - 2, q); }

/* ------------------------------------------------------------------ */
/* primes, factorisation, generator, psi                              */
/* ------------------------------------------------------------------ */

/* Deterministic Miller-Rabin: the first twelve primes as bases are
 * sufficient for every n < 3.3e24, hence for all 64-bit n. */
int orc_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n % bases[i] == 0) return n == bases[i];
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 12; ++i) {
        u64 x = orc_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/* Distinct prime factors of m by trial division: divide out 2, then odd d
 * while d*d <= rest; whenever the rest changes, stop early if it is prime.
 * Returns the number of distinct factors (entries beyond cap are dropped). */
int orc_prime_factors(u64 m, u64 *out, int cap)
{
    int k = 0;
    u64 rest = m;
    if (rest > 1 && rest % 2 == 0) {
        if (k < cap) out[k] = 2;
        ++k;
        while (rest % 2 == 0) rest /= 2;
    }
    if (rest > 1 && orc_is_prime(rest)) {
        if (k < cap) out[k] = rest;
        return k + 1;
    }
    for (u64 d = 3; rest > 1 && (u128)d * d <= rest; d += 2) {
        if (rest % d == 0) {
            if (k < cap) out[k] = d;
            ++k;
            while (rest % d == 0) rest /= d;
            if (rest > 1 && orc_is_prime(rest)) {
                if (k < cap) out[k] = rest;
                return k + 1;
            }
        }
    }
    if (rest > 1) {
        if (k < cap) out[k] = rest;
        ++k;
    }
    return k;
}

/* Smallest g >= 2 of multiplicative order q-1: g^{(q-1)/f} != 1 for every
 * prime f dividing q-1.  Returns 0 if q is not prime. */
u64 orc_smallest_generator(u64 q)
{
    u64 f[64];
    if (!orc_is_prime(q)) return 0;
    if (q == 2) return 1;
    int nf = orc_prime_factors(q - 1, f, 64);
    for (u64 g = 2; g < q; ++g) {
        int ok = 1;
        for (int i = 0; i < nf; ++i) {
            if (orc_powmod(g, (q - 1) / f[i], q) == 1) { ok = 0; break; }
        }
        if (ok) return g;
    }
    return 0;
}

/* psi = g^{(q-1)/(2N)}: a primitive 2N-th root of unity when 2N | q-1.
 * Returns 0 when q is not prime or 2N does not divide q-1. */
u64 orc_psi(u64 q, u64 N)
{
    if (N == 0 || q < 3 || (q - 1) % (2 * N) != 0) return 0;
    u64 g = orc_smallest_generator(q);
    if (g == 0) return 0;
    return orc_powmod(g, (q - 1) / (2 * N), q);
}

/* n-bit reversal of i */
u64 orc_bitrev(u64 i, int nbits)
{
    u64 r = 0;
    for (int b = 0; b < nbits; ++b) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

static int log2u(u64 N)
{
    int n = 0;
    while (((u64)1 << n) < N) ++n;
    return n;
}

/* ------------------------------------------------------------------ */
/* definitions, O(N^2)                                                */
/* ------------------------------------------------------------------ */

/* out[i] = sum_n a[n] psi^{n(2 brv(i)+1)} (Sec. III-A merged form, output in
 * the bit-reversed order of Algorithm 1). */
void orc_ntt_schoolbook(const u64 *a, u64 *out, u64 N, u64 q, u64 psi)
{
    int n = log2u(N);
    for (u64 i = 0; i < N; ++i) {
        u64 k = orc_bitrev(i, n);
        u64 root = orc_powmod(psi, 2 * k + 1, q);   /* psi^{2k+1} */
        u64 acc = 0, pw = 1;                        /* pw = root^n */
        for (u64 j = 0; j < N; ++j) {
            acc = addmod(acc, mulmod(a[j], pw, q), q);
            pw = mulmod(pw, root, q);
        }
        out[i] = acc;
    }
}

/* a[n] = N^{-1} sum_i out[i] psi^{-n(2 brv(i)+1)} */
void orc_intt_schoolbook(const u64 *A, u64 *out, u64 N, u64 q, u64 psi)
{
    int n = log2u(N);
    u64 psi_inv = orc_invmod(psi, q);
    u64 n_inv = orc_invmod(N % q, q);
    for (u64 j = 0; j < N; ++j) out[j] = 0;
    for (u64 i = 0; i < N; ++i) {
        u64 k = orc_bitrev(i, n);
        u64 root = orc_powmod(psi_inv, 2 * k + 1, q);
        u64 pw = 1;
        for (u64 j = 0; j < N; ++j) {
            out[j] = addmod(out[j], mulmod(A[i], pw, q), q);
            pw = mulmod(pw, root, q);
        }
    }
    for (u64 j = 0; j < N; ++j) out[j] = mulmod(out[j], n_inv, q);
}

/* c_k = sum_{i<=k} a_i b_{k-i} - sum_{i>k} a_i b_{N+k-i}   (Sec. III-A) */
void orc_negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *c, u64 N, u64 q)
{
    for (u64 k = 0; k < N; ++k) {
        u64 acc = 0;
        for (u64 i = 0; i <= k; ++i) acc = addmod(acc, mulmod(a[i], b[k - i], q), q);
        for (u64 i = k + 1; i < N; ++i) acc = submod(acc, mulmod(a[i], b[N + k - i], q), q);
        c[k] = acc;
    }
}

/* p(x) = sum_j a[j] x^j by Horner's rule */
u64 orc_eval(const u64 *a, u64 N, u64 x, u64 q)
{
    u64 acc = 0;
    for (u64 j = N; j-- > 0;) acc = addmod(mulmod(acc, x, q), a[j], q);
    return acc;
}

/* ------------------------------------------------------------------ */
/* fast transforms, O(N log N)                                        */
/* ------------------------------------------------------------------ */

/* Psi[i] = psi^{brv(i)} (Algorithm 1 input, Sec. III-C list) */
static void twiddles_bitrev(u64 *Psi, u64 N, u64 q, u64 root)
{
    int n = log2u(N);
    for (u64 i = 0; i < N; ++i) Psi[i] = orc_powmod(root, orc_bitrev(i, n), q);
}

/* Algorithm 1 (Cooley-Tukey), in place, natural order in, bit-reversed out.
 * Butterfly (Algorithm 2) on canonical values: V = a[k+t] Psi[m+j];
 * a[k] = a[k] + V; a[k+t] = a[k] - V. */
int orc_ntt_radix2(u64 *a, u64 N, u64 q, u64 psi)
{
    u64 *Psi = (u64 *)malloc(N * sizeof(u64));
    if (!Psi) return -1;
    twiddles_bitrev(Psi, N, q, psi);
    u64 t = N / 2;
    for (u64 m = 1; m < N; m *= 2) {
        for (u64 j = 0; j < m; ++j) {
            u64 w = Psi[m + j];
            for (u64 k = j * 2 * t; k < j * 2 * t + t; ++k) {
                u64 U = a[k];
                u64 V = mulmod(a[k + t], w, q);
                a[k] = addmod(U, V, q);
                a[k + t] = submod(U, V, q);
            }
        }
        t /= 2;
    }
    free(Psi);
    return 0;
}

/* Inverse of Algorithm 1 (Gentleman-Sande), in place: bit-reversed in,
 * natural order out, with Psi^{-1}[i] = psi^{-brv(i)} merged into the stages
 * and a final scaling by N^{-1}.  Stage order is the exact reverse of
 * Algorithm 1; each butterfly undoes the forward one up to a factor 2:
 *   U = a[k]; V = a[k+t]; a[k] = U + V; a[k+t] = (U - V) Psi^{-1}[m+j]. */
int orc_intt_radix2(u64 *a, u64 N, u64 q, u64 psi)
{
    u64 *Pinv = (u64 *)malloc(N * sizeof(u64));
    if (!Pinv) return -1;
    twiddles_bitrev(Pinv, N, q, orc_invmod(psi, q));
    u64 t = 1;
    for (u64 m = N / 2; m >= 1; m /= 2) {
        for (u64 j = 0; j < m; ++j) {
            u64 w = Pinv[m + j];
            for (u64 k = j * 2 * t; k < j * 2 * t + t; ++k) {
                u64 U = a[k];
                u64 V = a[k + t];
                a[k] = addmod(U, V, q);
                a[k + t] = mulmod(submod(U, V, q), w, q);
            }
        }
        t *= 2;
    }
    u64 n_inv = orc_invmod(N % q, q);
    for (u64 k = 0; k < N; ++k) a[k] = mulmod(a[k], n_inv, q);
    free(Pinv);
    return 0;
}

void orc_pointwise(const u64 *a, const u64 *b, u64 *c, u64 n, u64 q)
{
    for (u64 i = 0; i < n; ++i) c[i] = mulmod(a[i], b[i], q);
}

/* ------------------------------------------------------------------ */
/* batched driver over [batch][L][N], threaded over limbs             */
/* ------------------------------------------------------------------ */
struct batch_job {
    u64 *data;
    u64 N;
    const u64 *primes;
    const u64 *psis;
    u64 L, batch;
    int dir;
    int stride, first;
    int err;
};

static void *batch_worker(void *arg)
{
    struct batch_job *j = (struct batch_job *)arg;
    u64 total = j->L * j->batch;
    for (u64 idx = (u64)j->first; idx < total; idx += (u64)j->stride) {
        u64 l = idx % j->L;
        u64 *limb = j->data + idx * j->N;
        int rc = j->dir > 0 ? orc_ntt_radix2(limb, j->N, j->primes[l], j->psis[l])
                            : orc_intt_radix2(limb, j->N, j->primes[l], j->psis[l]);
        if (rc) j->err = rc;
    }
    return 0;
}

/* In-place forward (dir > 0) or inverse (dir < 0) transform of every limb of
 * data[batch][L][N] with prime primes[l]; psi per prime is derived with
 * orc_psi.  Uses up to `threads` POSIX threads.  Returns 0, or -1 on a bad
 * argument (non-prime, q != 1 mod 2N), or -2 on allocation failure. */
int orc_ntt_batch(u64 *data, u64 N, const u64 *primes, u64 L, u64 batch, int dir, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    u64 *psis = (u64 *)malloc(L * sizeof(u64));
    if (!psis) return -2;
    for (u64 l = 0; l < L; ++l) {
        psis[l] = orc_psi(primes[l], N);
        if (psis[l] == 0) { free(psis); return -1; }
    }
    struct batch_job jobs[256];
    pthread_t tid[256];
    int created[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].data = data; jobs[t].N = N; jobs[t].primes = primes; jobs[t].psis = psis;
        jobs[t].L = L; jobs[t].batch = batch; jobs[t].dir = dir;
        jobs[t].stride = threads; jobs[t].first = t; jobs[t].err = 0;
        created[t] = 0;
    }
    if (threads == 1) {
        batch_worker(&jobs[0]);
    } else {
        for (int t = 0; t < threads; ++t) {
            if (pthread_create(&tid[t], 0, batch_worker, &jobs[t]) == 0) created[t] = 1;
            else batch_worker(&jobs[t]);
        }
        for (int t = 0; t < threads; ++t) if (created[t]) pthread_join(tid[t], 0);
    }
    int err = 0;
    for (int t = 0; t < threads; ++t) if (jobs[t].err) err = -2;
    free(psis);
    return err;
}

/* c[b][l][:] = a[b][l][:] * b[b][l][:] mod primes[l] */
void orc_pointwise_batch(const u64 *a, const u64 *b, u64 *c, u64 N, const u64 *primes, u64 L, u64 batch)
{
    for (u64 bb = 0; bb < batch; ++bb)
        for (u64 l = 0; l < L; ++l) {
            u64 off = (bb * L + l) * N;
            orc_pointwise(a + off, b + off, c + off, N, primes[l]);
        }
}
