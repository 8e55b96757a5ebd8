"""CPU model of the pass kernels' index math and lazy arithmetic (test only).

Mirrors paper_2012_01968_gb300/csrc/ntt_pass.cuh and arith.cuh: the tile
geometry, item decomposition, round schedule, twiddle indices (table and
on-the-fly), the lazy Shoup product with its 3-partial-product quotient, the
final reduction and the range bookkeeping, with every value checked against the
bound the kernel assumes (below 2^64 and below X q).  Used to check the
kernel design against the oracle on the CPU before it runs on a GPU.
"""
from __future__ import annotations

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def brv(i, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (i & 1)
        i >>= 1
    return r


def shoup_lazy(y, w, wp, q):
    assert 0 <= y <= M64 and 0 <= w < q
    yl, yh = y & M32, y >> 32
    qhat = yh * (wp >> 32) + ((yh * (wp & M32)) >> 32) + ((yl * (wp >> 32)) >> 32)
    assert qhat <= M64
    # the kernel forms the low word of y*w + qhat*(2^64 - q) from 32-bit pieces
    nq = (1 << 64) - q
    lo = ((y & M32) * (w & M32) + (qhat & M32) * (nq & M32)) & M64
    rh = ((lo >> 32) + yl * (w >> 32) + yh * (w & M32) + (qhat & M32) * (nq >> 32) + (qhat >> 32) * (nq & M32)) & M32
    r = (rh << 32) | (lo & M32)
    assert r == (y * w - qhat * q) & M64
    assert r < 4 * q and r % q == (y * w) % q
    return r


def reduce2(x, q, rc, rsh):
    """x mod q into [0, 2q) for x < 16q from the top 32 bits of x (arith.cuh)."""
    assert 0 <= x < 16 * q and rsh == q.bit_length() - 28 and 5 <= rsh <= 32
    xs = x >> rsh
    assert xs <= M32
    kq = ((xs * rc) >> 32) >> 27
    r = x - kq * q
    assert 0 <= r < 2 * q
    return r


def canon(x, X, q, rc, rsh):
    assert x < X * q
    if X > 4:
        x = reduce2(x, q, rc, rsh)
        return csub(x, q)
    if X > 2:
        x = csub(x, 2 * q)
    if X > 1:
        x = csub(x, q)
    return x


def reduction_constants(q):
    """(rc, rsh) = (floor(2^(k+31) / q), k - 28), k the bit length of q."""
    k = q.bit_length()
    rc = (1 << (k + 31)) // q
    assert (1 << 31) <= rc <= M32
    return rc, k - 28


def ct_reduces(X):
    return X + 4 > 16


def ct_next(X):
    return 12 if ct_reduces(X) else X + 4


def gs_reduces(X):
    return 2 * X > 8


def gs_next(X):
    return 8 if gs_reduces(X) else (2 * X if 2 * X > 4 else 4)


def csub(x, c):
    """x in [0, 2c) -> [0, c) the way arith.cuh decides it for 64-bit words:
    by the sign bit of the wrapped difference x - c (valid for c <= 2^63)."""
    assert 0 <= x < 2 * c and c <= 1 << 63
    d = (x - c) & M64
    r = x if d >> 63 else d
    assert r == (x - c if x >= c else x)
    return r


def ct_after(X, k):
    for _ in range(k):
        X = ct_next(X)
    return X


def gs_after(X, k):
    for _ in range(k):
        X = gs_next(X)
    return X


def rounds(P, KMAX):
    nr = (P + KMAX - 1) // KMAX
    sizes = [P // nr + (1 if r < P % nr else 0) for r in range(nr)]
    starts = [sum(sizes[:r]) for r in range(nr)]
    return sizes, starts


def tw_slot(j, sl, K0, k):
    """Table slot of butterfly j of a stage (mirror of tw_slot in ntt_pass.cuh)."""
    return (j >> sl << sl) | ((j & ((1 << k) - 1)) << K0) | ((j >> k) & ((1 << K0) - 1))


def stage_slot_params(n, p1, s, KMAX=4):
    """(sl, K0, k) of stage s in the pass that holds it (mirror of plan.h)."""
    if n <= 12:
        s0, P = 0, n
    elif s < p1:
        s0, P = 0, p1
    else:
        s0, P = p1, n - p1
    sl = s - s0
    sizes, starts = rounds(P, KMAX)
    for sz, st in zip(sizes, starts):
        if sl < st + sz:
            return sl, st, sl - st
    return sl, 0, sl


def swz(w):
    return w ^ (((w >> 4) & 7) << 1)


class PrimeTables:
    """Tables for one prime, built as the plan builds them."""

    def __init__(self, q, psi, n, p1, ots):
        N = 1 << n
        self.q, self.n, self.N = q, n, N
        pw = [1] * N
        for e in range(1, N):
            pw[e] = pw[e - 1] * psi % q
        fwd = lambda e: pw[e]
        inv = lambda e: 1 if e == 0 else q - pw[N - e]
        comp = lambda w: (w << 64) // q
        self.tw_len = N >> ots
        self.tw = [None] * self.tw_len
        self.tw[0] = (1, comp(1))
        s = 0
        while (1 << s) < self.tw_len:
            sl, K0, k = stage_slot_params(n, p1, s)
            for j in range(1 << s):
                w = fwd(brv((1 << s) + j, n))
                self.tw[(1 << s) + tw_slot(j, sl, K0, k)] = (w, comp(w))
            s += 1
        self.rc, self.rsh = reduction_constants(q)
        ninv = pow(N, q - 2, q)
        self.ninv = (ninv, comp(ninv))
        w1 = fwd(brv(1, n)) if N >= 2 else 1
        self.w1ninv = (w1 * ninv % q, comp(w1 * ninv % q))
        p2 = n - p1
        R = 1 << p2
        self.ota_f = [(1, comp(1))] * R
        self.ota_i = [(1, comp(1))] * R
        for sl in range(p2):
            _, K0, k = stage_slot_params(n, p1, p1 + sl)
            for j in range(1 << sl):
                e = brv(j, sl) << (n - sl)
                slot = (1 << sl) + tw_slot(j, sl, K0, k)
                self.ota_f[slot] = (fwd(e), comp(fwd(e)))
                self.ota_i[slot] = (inv(e), comp(inv(e)))
        s0 = p1
        self.otb_f = [None] * (p2 << s0)
        self.otb_i = [None] * (p2 << s0)
        for sl in range(p2):
            for u in range(1 << s0):
                s = s0 + sl
                e = (2 * brv(u, s0) + 1) << (n - 1 - s)
                self.otb_f[(sl << s0) + u] = (fwd(e), comp(fwd(e)))
                self.otb_i[(sl << s0) + u] = (inv(e), comp(inv(e)))


def run_pass(data, T: PrimeTables, *, P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM, s0):
    """Apply one pass to one limb (list of ints) in place, tile by tile."""
    n, q = T.n, T.q
    N = 1 << n
    R, C = 1 << P, 1 << LOGC
    b = n - s0 - P
    nb = n - s0
    TILE = R * C
    sizes, starts = rounds(P, KMAX)
    NR = len(sizes)
    tiles = N >> (P + LOGC)
    seen = [0] * N
    q4 = 4 * q
    for tile in range(tiles):
        if ROWS:
            u_base, l0 = tile * C, 0
        else:
            per_u = (1 << b) >> LOGC
            u_base, l0 = tile // per_u, (tile % per_u) * C
        sm = [None] * TILE
        # load
        for i in range(TILE // 2):
            if ROWS:
                g = (u_base << P) + 2 * i
                w = 2 * i
            else:
                VPR = C // 2
                v, cv = i // VPR, i % VPR
                g = (u_base << nb) + l0 + (v << b) + 2 * cv
                w = v * C + 2 * cv
            assert 0 <= g and g + 1 < N
            sw = swz(w)
            assert sw % 2 == 0 and sw + 1 < TILE
            sm[sw], sm[sw + 1] = data[g], data[g + 1]
            seen[g] += 1
            seen[g + 1] += 1
        order = range(NR) if FWD else range(NR - 1, -1, -1)
        for r in order:
            KR, K0 = sizes[r], starts[r]
            E = 1 << KR
            NLO = P - K0 - KR
            if FWD:
                XR = ct_after(XIN, K0)
            else:
                XR = gs_after(XIN, P - K0 - KR)
            items = C << (P - KR)
            canon_here = FINAL and ((FWD and r == NR - 1) or ((not FWD) and r == 0))
            for it in range(items):
                if ROWS:
                    lo = it & ((1 << NLO) - 1)
                    hi = (it >> NLO) & ((1 << K0) - 1)
                    cc = it >> (NLO + K0)
                    u = u_base + cc
                else:
                    cc = it & (C - 1)
                    lo = (it >> LOGC) & ((1 << NLO) - 1)
                    hi = it >> (LOGC + NLO)
                    u = u_base
                vbase = (hi << (P - K0)) | lo
                idx = []
                for i in range(E):
                    v = vbase | (i << NLO)
                    w = cc * R + v if ROWS else v * C + cc
                    idx.append(swz(w))
                x = [sm[j] for j in idx]
                X = XR
                ks = range(KR) if FWD else range(KR - 1, -1, -1)
                if not FWD:
                    # the inverse applies gs_next per executed stage, in order
                    Xs = {}
                    Xc = XR
                    for k in ks:
                        Xs[k] = Xc
                        Xc = gs_next(Xc)
                for k in ks:
                    half = E >> (k + 1)
                    sl = K0 + k
                    ot = sl >= P - OTS
                    if FWD:
                        assert X + 4 <= 16 or ct_reduces(X)
                    else:
                        X = Xs[k]
                        assert X <= 8
                    if (not FWD) and HAS_S0 and K0 == 0 and k == 0:
                        for i in range(half):
                            a, bb = x[i], x[i + half]
                            Xq = X * q
                            d = bb + Xq - a
                            assert a < Xq and bb < Xq
                            x[i] = shoup_lazy(a + bb, T.ninv[0], T.ninv[1], q)
                            x[i + half] = shoup_lazy(d, T.w1ninv[0], T.w1ninv[1], q)
                        continue
                    for pre in range(1 << k):
                        jlo = (pre << K0) | hi
                        if ot:
                            B = (T.otb_f if FWD else T.otb_i)[(sl << s0) + u]
                            A = (T.ota_f if FWD else T.ota_i)[(1 << sl) + jlo]
                        else:
                            if FWD:
                                ix = (1 << (s0 + sl)) + (u << sl) + jlo if not TW_SMEM else (1 << sl) + jlo
                            else:
                                j = (u << sl) + jlo if not TW_SMEM else jlo
                                ix = ((2 << (s0 + sl)) - 1 - j) if not TW_SMEM else ((2 << sl) - 1 - j)
                            assert 0 <= ix < (T.tw_len if not TW_SMEM else R)
                            tw = T.tw[ix]
                        for i in range(half):
                            ia, ib = pre * 2 * half + i, pre * 2 * half + i + half
                            a, bb = x[ia], x[ib]
                            if FWD:
                                assert a < X * q and bb < X * q
                                if ct_reduces(X):
                                    a = csub(a, 8 * q)
                                t = shoup_lazy(shoup_lazy(bb, *B, q), *A, q) if ot else shoup_lazy(bb, tw[0], tw[1], q)
                                x[ia] = a + t
                                x[ib] = a + q4 - t
                                assert x[ia] <= M64 and x[ib] <= M64
                            else:
                                Xq = X * q
                                assert a < Xq and bb < Xq
                                d = (a + Xq - bb) if ot else (bb + Xq - a)
                                s = a + bb
                                if gs_reduces(X):
                                    s = csub(s, 8 * q)
                                x[ia] = s
                                x[ib] = shoup_lazy(shoup_lazy(d, *B, q), *A, q) if ot else shoup_lazy(d, tw[0], tw[1], q)
                    if FWD:
                        X = ct_next(X)
                if canon_here:
                    if FWD:
                        x = [canon(v, ct_after(XIN, P), q, T.rc, T.rsh) for v in x]
                    else:
                        x = [canon(v, 4 if HAS_S0 else gs_after(XIN, P), q, T.rc, T.rsh) for v in x]
                for j, v in zip(idx, x):
                    sm[j] = v
        # store
        for i in range(TILE // 2):
            if ROWS:
                g, w = (u_base << P) + 2 * i, 2 * i
            else:
                VPR = C // 2
                v, cv = i // VPR, i % VPR
                g = (u_base << nb) + l0 + (v << b) + 2 * cv
                w = v * C + 2 * cv
            sw = swz(w)
            data[g], data[g + 1] = sm[sw], sm[sw + 1]
    assert all(s == 1 for s in seen), "every word loaded exactly once"


def split(n):
    if n <= 12:
        return n, 0
    p2 = (n + 1) // 2
    return n - p2, p2


def logc_rows(p2):
    return min(5, 12 - p2)


# (p1, log2 rows per row tile) of the two-pass geometries 0, 1, 2 (n = 13 .. 17)
GEOMETRIES = {13: [(6, 5), (6, 4), (7, 6)], 14: [(7, 5), (7, 4), (6, 4)], 15: [(7, 4), (7, 3), (8, 5)],
              16: [(8, 4), (8, 3), (7, 3)], 17: [(8, 3), (8, 2), (7, 2)]}


def transform(a, q, psi, n, fwd, ots=0, geometry=0):
    """Whole transform as the library dispatches it (one limb)."""
    data = [int(v) for v in a]
    p1, p2 = split(n)
    if p2 and geometry:
        p1, LRg = GEOMETRIES[n][geometry]
        p2 = n - p1
    if p2 == 0:
        T = PrimeTables(q, psi, n, n, 0)
        run_pass(data, T, P=n, LOGC=0, KMAX=4, ROWS=True, FWD=fwd, XIN=1, FINAL=True, HAS_S0=True,
                 OTS=0, TW_SMEM=False, s0=0)
        return data
    T = PrimeTables(q, psi, n, p1, ots)
    LR = LRg if geometry else logc_rows(p2)
    if fwd:
        run_pass(data, T, P=p1, LOGC=4, KMAX=4, ROWS=False, FWD=True, XIN=1, FINAL=False, HAS_S0=True,
                 OTS=0, TW_SMEM=True, s0=0)
        run_pass(data, T, P=p2, LOGC=LR, KMAX=4, ROWS=True, FWD=True, XIN=ct_after(1, p1), FINAL=True,
                 HAS_S0=False, OTS=ots, TW_SMEM=False, s0=p1)
    else:
        run_pass(data, T, P=p2, LOGC=LR, KMAX=4, ROWS=True, FWD=False, XIN=1, FINAL=False, HAS_S0=False,
                 OTS=ots, TW_SMEM=False, s0=p1)
        run_pass(data, T, P=p1, LOGC=4, KMAX=4, ROWS=False, FWD=False, XIN=gs_after(1, p2), FINAL=True,
                 HAS_S0=True, OTS=0, TW_SMEM=True, s0=0)
    return data


def fused_geometry(n):
    """(UA, UB, threads) of the fused kernel for N = 2^n, forward direction."""
    p1, p2 = split(n)
    lr = logc_rows(p2)
    UC, UR = (1 << p2) // 16, (1 << p1) >> lr
    return UC, UR


def high_radix_transform(a, q, psi, n, k, fwd):
    """The register-based high-radix organisation's index maps (one launch per
    group of k stages; item = 2^k elements spaced t apart; natural-order table),
    with exact modular butterflies."""
    N = 1 << n
    pw = [1] * N
    for e in range(1, N):
        pw[e] = pw[e - 1] * psi % q
    tw = [pw[brv(i, n)] for i in range(N)]          # Psi[i] = psi^brv(i), natural order
    ninv = pow(N, q - 2, q)
    d = [int(v) for v in a]
    groups = (n + k - 1) // k
    order = range(groups) if fwd else range(groups - 1, -1, -1)
    for g in order:
        s0 = g * k
        kk = min(k, n - s0)
        nb = n - s0 - kk
        for m in range(N >> kk):
            b, j = m >> nb, m & ((1 << nb) - 1)
            base = (b << (n - s0)) + j
            idx = [base + (i << nb) for i in range(1 << kk)]
            x = [d[i] for i in idx]
            rs = range(kk) if fwd else range(kk - 1, -1, -1)
            for r in rs:
                h = 1 << (kk - 1 - r)
                s = s0 + r
                for grp in range(1 << r):
                    for i in range(h):
                        lo, hi = grp * 2 * h + i, grp * 2 * h + i + h
                        if fwd:
                            w = tw[(1 << s) + (b << r) + grp]
                            v = x[hi] * w % q
                            x[lo], x[hi] = (x[lo] + v) % q, (x[lo] - v) % q
                        elif s == 0:
                            # stage 0 with N^{-1} folded in: (x + y) / N and (y - x) Psi[1] / N
                            u, v = x[lo], x[hi]
                            x[lo] = (u + v) * ninv % q
                            x[hi] = (v - u) * tw[1] % q * ninv % q
                        else:
                            jj = (b << r) + grp
                            w = tw[(2 << s) - 1 - jj]      # -Psi^{-1}[2^s + jj]
                            u, v = x[lo], x[hi]
                            x[lo] = (u + v) % q
                            x[hi] = (v - u) * w % q
            for i, v in zip(idx, x):
                d[i] = v
    return d
