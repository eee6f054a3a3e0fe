// Stage kernels of the 3D r2c / c2r transform (P3DFFT paper, Sect. 2 and
// Sect. 3.3): each launch applies one batched 1D transform to every line of
// the volume along one dimension.
//
// One CTA owns a tile of B lines (B a power of two).  The tile is read from
// HBM into shared memory (element e of tile line l at s[e * LDB + l]), with
// the op's pre-processing and any change of pencil orientation folded into
// the load addressing; a mixed-radix Stockham FFT (radix 2, 3, 4, 5, 7, 8, 16,
// register butterflies, twiddles from an FP64-derived table) runs in shared
// memory; the tile is written back with the op's post-processing folded into
// the store addressing.  Lines whose elements are contiguous in HBM are read
// and written with lanes walking the elements; strided lines with lanes
// walking adjacent lines, so every global access is coalesced.  This is the
// paper's "transpose inside the FFT call" alternative (Sect. 3.3) done in
// shared memory, replacing the pack / all-to-all / unpack / local-transpose
// sequence between pencils.
#include <cstddef>

#include "p3_dft.cuh"
#include "p3_internal.h"

namespace p3 {
namespace {

// ---------------------------------------------------------------------------
// One Stockham (autosort, decimation in time) pass of radix R over n points
// of every tile line, from buffer src to buffer dst (ping-pong, so each
// butterfly is read, transformed and written at once and only R values are
// live).  Butterfly j reads elements j + r n/R, multiplies by
// exp(-2 pi i (j mod Ns) r / (Ns R)), does a size-R DFT and writes
// (j / Ns) Ns R + (j mod Ns) + r Ns.  Thread t of a line takes butterflies
// t, t + tpl, ...; j / Ns and j mod Ns are updated incrementally.
// ---------------------------------------------------------------------------
template <class C, class T, int R, bool SWAP = false>
__device__ __forceinline__ void pass_pp(const C* src, C* dst, int LDB, int l, int t, int tpl, int n, int Ns,
                                        const PassConsts& c, const C* tw)
{
    const int nb = n / R;
    const int istride = nb * LDB, ostride = Ns * LDB;  // slots between a butterfly's inputs / outputs
    const int tstep = c.tstep;                         // table index of one unit of j mod Ns
    int q = (int)(((unsigned long long)(unsigned)t * c.pm) >> c.ps), rr = t - q * Ns;
    const int dq = c.dq, dr = c.dr;
    for (int j = t; j < nb; j += tpl) {
        C v[R];
        const C* sp = src + j * LDB + l;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = SWAP ? swp(sp[r * istride]) : sp[r * istride];
        if (rr) {
            // exp(-2 pi i rr r / (Ns R)) = tw[rr r (n / (Ns R)) ts], the index
            // kept as a running 32-bit sum
            const int k = rr * tstep;
            int idx = k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                v[r] = mul(v[r], ldg(tw + idx));
                idx += k;
            }
        }
        Dft<C, T, R>::run(v);
        C* dp = dst + (q * Ns * R + rr) * LDB + l;
#pragma unroll
        for (int r = 0; r < R; ++r) dp[r * ostride] = v[r];
        rr += dr;
        q += dq;
        if (rr >= Ns) {
            rr -= Ns;
            ++q;
        }
    }
}

// All passes; the data starts in buf0 and the returned buffer holds the
// result.  swap_in: the first pass swaps real and imaginary parts of its
// inputs (the inverse transform as swp(DFT(swp(.)))).
template <class C, class T, bool SWAP>
__device__ __forceinline__ void pass_any(int R, const C* src, C* dst, int LDB, int l, int t, int tpl, int n, int Ns,
                                         const PassConsts& c, const C* tw)
{
    switch (R) {
    case 16: pass_pp<C, T, 16, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    case 8: pass_pp<C, T, 8, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    case 4: pass_pp<C, T, 4, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    case 2: pass_pp<C, T, 2, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    case 3: pass_pp<C, T, 3, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    case 5: pass_pp<C, T, 5, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    case 7: pass_pp<C, T, 7, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
    default:
        // composite radices (FP32 plans only; see the plan's factorisation)
        if constexpr (sizeof(T) == 4) {
            switch (R) {
            case 6: if constexpr (6 <= P3_GEN_MAXCR) pass_pp<C, T, 6, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 9: if constexpr (9 <= P3_GEN_MAXCR) pass_pp<C, T, 9, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 10: if constexpr (10 <= P3_GEN_MAXCR) pass_pp<C, T, 10, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 12: if constexpr (12 <= P3_GEN_MAXCR) pass_pp<C, T, 12, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 14: if constexpr (14 <= P3_GEN_MAXCR) pass_pp<C, T, 14, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 15: if constexpr (15 <= P3_GEN_MAXCR) pass_pp<C, T, 15, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 18: if constexpr (18 <= P3_GEN_MAXCR) pass_pp<C, T, 18, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 20: if constexpr (20 <= P3_GEN_MAXCR) pass_pp<C, T, 20, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 21: if constexpr (21 <= P3_GEN_MAXCR) pass_pp<C, T, 21, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 24: if constexpr (24 <= P3_GEN_MAXCR) pass_pp<C, T, 24, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 25: if constexpr (25 <= P3_GEN_MAXCR) pass_pp<C, T, 25, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 27: if constexpr (27 <= P3_GEN_MAXCR) pass_pp<C, T, 27, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            case 28: if constexpr (28 <= P3_GEN_MAXCR) pass_pp<C, T, 28, SWAP>(src, dst, LDB, l, t, tpl, n, Ns, c, tw); break;
            default: break;
            }
        }
        break;
    }
}

template <class C, class T>
__device__ __forceinline__ C* run_passes(C* buf0, C* buf1, int LDB, int l, int t, int tpl, bool act, int n,
                                         int npass, const int* rad, const PassConsts* pc, const C* tw,
                                         bool swap_in = false)
{
    int Ns = 1;
    C* src = buf0;
    C* dst = buf1;
    for (int p = 0; p < npass; ++p) {
        const int R = rad[p];
        if (act) {
            if (p == 0 && swap_in)
                pass_any<C, T, true>(R, src, dst, LDB, l, t, tpl, n, Ns, pc[p], tw);
            else
                pass_any<C, T, false>(R, src, dst, LDB, l, t, tpl, n, Ns, pc[p], tw);
        }
        __syncthreads();
        Ns *= R;
        C* tmp = src;
        src = dst;
        dst = tmp;
    }
    return src;
}

__device__ __forceinline__ long long line_base(const LineMap& m, long long L)
{
    if (m.pm) {  // L < 2^31: quotient by multiply-high (line_magic)
        const unsigned u = (unsigned)L;
        const unsigned q = (unsigned)(((unsigned long long)u * m.pm) >> m.ps);
        const unsigned r = u - q * (unsigned)m.per;
        return (long long)q * m.gstride + (long long)r * m.lstride;
    }
    return (L / m.per) * m.gstride + (L % m.per) * m.lstride;
}

// Value placed in shared-memory slot e of a line before the FFT (the op
// fixed at compile time).
template <int OP, bool BLUE, class C, class T>
__device__ __forceinline__ C load_value(const StageArgs& a, long long base, int e)
{
    const long long es = a.in.es;
    C v;
    switch (OP) {
    case OP_R2C_HALF: {  // z[j] = f[2j] + i f[2j+1]; rows are contiguous
        const T* f = static_cast<const T*>(a.src);
        v = *reinterpret_cast<const C*>(f + base + 2 * (long long)e);
        break;
    }
    case OP_C2R_HALF: {
        // Z[k] = (F[k] + conj F[n-k]) + i (F[k] - conj F[n-k]) exp(+2 pi i k / Nx),
        // n = Nx/2, with the imaginary parts of F[0] and F[n] dropped.
        const C* F = static_cast<const C*>(a.src);
        const int n = a.nfft;
        C A = F[base + (long long)e * es];
        C B = cnj(F[base + (long long)(n - e) * es]);
        if (e == 0) {
            A.y = (T)0;
            B.y = (T)0;
        }
        const C ze = add(A, B);
        const C zo = mul(sub(A, B), cnj(ldg(static_cast<const C*>(a.tw2) + e)));
        v = swp(mk<C>(ze.x - zo.y, ze.y + zo.x));
        break;
    }
    case OP_DCT1: {  // even extension y[e] = x[e] (e <= M), x[2M - e] (e > M)
        const C* X = static_cast<const C*>(a.src);
        const int M = a.n_in - 1;
        const int src = e <= M ? e : 2 * M - e;
        v = X[base + (long long)src * es];
        break;
    }
    case OP_DST1: {  // odd extension y = (0, x[0..n-1], 0, -x[n-1..0])
        const C* X = static_cast<const C*>(a.src);
        const int n = a.n_in;
        if (e == 0 || e == n + 1) {
            v = mk<C>((T)0, (T)0);
        } else if (e <= n) {
            v = X[base + (long long)(e - 1) * es];
        } else {
            const C u = X[base + (long long)(2 * n + 1 - e) * es];
            v = mk<C>(-u.x, -u.y);
        }
        break;
    }
    default: {  // OP_C2C, OP_COPY
        const C* X = static_cast<const C*>(a.src);
        v = X[base + (long long)e * es];
        if (a.sign > 0) v = swp(v);
        break;
    }
    }
    if constexpr (BLUE) v = mul(v, ldg(static_cast<const C*>(a.chirp) + e));
    return v;
}

// Fills slots e0, e0 + de, ... (< nload) of line l from its input at base:
// KB loads of a thread are issued before any of them is stored, so their
// latencies overlap instead of adding up; slots at or past nfill are zero.
template <int OP, bool BLUE, class C, class T>
__device__ __forceinline__ void load_elems(const StageArgs& a, C* s0, int LDB, int l, long long base, int e0, int de,
                                           int nload, int nfill)
{
    constexpr int KB = sizeof(T) == 4 ? 8 : 4;
    const C zero = mk<C>((T)0, (T)0);
    for (int eb = e0; eb < nload; eb += de * KB) {
        C w[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            const int e = eb + de * k;
            w[k] = e < nfill ? load_value<OP, BLUE, C, T>(a, base, e) : zero;
        }
#pragma unroll
        for (int k = 0; k < KB; ++k)
            if (eb + de * k < nload) s0[(eb + de * k) * LDB + l] = w[k];
    }
}

template <bool BLUE, class C, class T>
__device__ __forceinline__ void load_line(const StageArgs& a, C* s0, int LDB, int l, long long base, int e0, int de,
                                          int nload, int nfill)
{
    switch (a.op) {
    case OP_R2C_HALF: load_elems<OP_R2C_HALF, BLUE, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill); break;
    case OP_C2R_HALF: load_elems<OP_C2R_HALF, BLUE, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill); break;
    case OP_DCT1: load_elems<OP_DCT1, BLUE, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill); break;
    case OP_DST1: load_elems<OP_DST1, BLUE, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill); break;
    default: load_elems<OP_C2C, BLUE, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill); break;
    }
}

// Odd real rows in pairs (the two-for-one real transform): line L of a
// pair op holds real rows 2L and 2L + 1 (the second absent, i.e. zero, when
// 2L + 1 = nrows), with bases b0 and b1 in the input (load) or output
// (store).
//
// Forward load: slot e = f1[e] + i f2[e].
// Inverse load: for k < H the half spectra give Z[k] = X1[k] + i X2[k] and
// Z[N-k] = conj X1[k] + i conj X2[k] (k >= 1; N odd, so k and N - k cover
// every bin once; the imaginary parts of X1[0] and X2[0] are dropped), swapped
// for the inverse FFT.  Then Re and Im of the inverse transform are the
// weighted-real C2R of X1 and of X2 (Sect. 3.2's complex-to-real transform).
template <int OP, bool BLUE, class C, class T>
__device__ __forceinline__ void pair_load(const StageArgs& a, C* s0, int LDB, int l, long long b0, long long b1,
                                          bool has2, int e0, int de, int nload, int nfill)
{
    const long long es = a.in.es;
    const C zero = mk<C>((T)0, (T)0);
    const C* chirp = static_cast<const C*>(a.chirp);
    if constexpr (OP == OP_R2C_PAIR) {
        constexpr int KB = sizeof(T) == 4 ? 8 : 4;
        const T* f = static_cast<const T*>(a.src);
        for (int eb = e0; eb < nload; eb += de * KB) {
            C w[KB];
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                const int e = eb + de * k;
                w[k] = zero;
                if (e < nfill) {
                    w[k].x = f[b0 + e * es];
                    if (has2) w[k].y = f[b1 + e * es];
                }
            }
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                const int e = eb + de * k;
                if (e < nload) s0[e * LDB + l] = (BLUE && e < nfill) ? mul(w[k], ldg(chirp + e)) : w[k];
            }
        }
    } else {  // OP_C2R_PAIR: k < H = n_in
        constexpr int KB = sizeof(T) == 4 ? 4 : 2;
        const C* F = static_cast<const C*>(a.src);
        const int H = a.n_in, N = a.nfft;
        for (int kb = e0; kb < H; kb += de * KB) {
            C A[KB], Bv[KB];
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                const int k = kb + de * u;
                A[u] = zero;
                Bv[u] = zero;
                if (k < H) {
                    A[u] = F[b0 + k * es];
                    if (has2) Bv[u] = F[b1 + k * es];
                }
            }
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                const int k = kb + de * u;
                if (k >= H) continue;
                if (k == 0) {
                    A[u].y = (T)0;
                    Bv[u].y = (T)0;
                }
                C zk = swp(mk<C>(A[u].x - Bv[u].y, A[u].y + Bv[u].x));
                if constexpr (BLUE) zk = mul(zk, ldg(chirp + k));
                s0[k * LDB + l] = zk;
                if (k > 0) {
                    C zm = swp(mk<C>(A[u].x + Bv[u].y, Bv[u].x - A[u].y));
                    if constexpr (BLUE) zm = mul(zm, ldg(chirp + (N - k)));
                    s0[(N - k) * LDB + l] = zm;
                }
            }
        }
        for (int e = nfill + e0; e < nload; e += de) s0[e * LDB + l] = zero;  // Bluestein padding
    }
}

// Forward store: X1[k] = (Z[k] + conj Z[N-k]) / 2 and X2[k] = -i (Z[k] -
// conj Z[N-k]) / 2 for k < H.  Inverse store: f1[j] = Re z[j], f2[j] = Im z[j].
template <int OP, bool BLUE, class C, class T>
__device__ __forceinline__ void pair_store(const StageArgs& a, const C* sl, int LDB, long long b0, long long b1,
                                           bool has2, int e0, int de)
{
    const long long es = a.out.es;
    const C* chirp = static_cast<const C*>(a.chirp);
    auto res = [&](int k) -> C {
        C v = sl[k * LDB];
        if constexpr (BLUE) v = mul(ldg(chirp + k), swp(v));
        return v;
    };
    if constexpr (OP == OP_R2C_PAIR) {
        const int N = a.nfft;
        C* X = static_cast<C*>(a.dst);
        for (int k = e0; k < a.n_out; k += de) {
            const C zk = res(k), zm = res(k == 0 ? 0 : N - k);
            X[b0 + k * es] = mk<C>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
            if (has2) X[b1 + k * es] = mk<C>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
        }
    } else {  // OP_C2R_PAIR
        T* f = static_cast<T*>(a.dst);
        for (int j = e0; j < a.n_out; j += de) {
            const C w = swp(res(j));
            f[b0 + j * es] = w.x;
            if (has2) f[b1 + j * es] = w.y;
        }
    }
}

// FP32 X stages whose rows lie one after another walk each tile's values as
// one run (1), or row by row with a warp per row (0).  FP64 stages, bound by
// the FP64 pipe, keep the row-by-row walk.
#ifndef P3_GEN_FLAT
#define P3_GEN_FLAT 1
#endif

// Ops whose load is a plain copy of one complex value (no pre-processing
// beyond the inverse's real/imaginary swap): their tiles are filled by
// asynchronous copies straight into shared memory, all of a thread's copies
// in flight at once and no registers held for them.
#ifndef P3_GEN_CPASYNC
#define P3_GEN_CPASYNC 1
#endif
__device__ __forceinline__ bool direct_load(const StageArgs& a)
{
    return P3_GEN_CPASYNC && !a.blue &&
           (a.op == OP_C2C || a.op == OP_COPY || a.op == OP_R2C_HALF || a.op == OP_C2R_HALF);
}

template <class C, class T>
__device__ __forceinline__ const C* direct_src(const StageArgs& a, long long base, int e)
{
    if (a.op == OP_R2C_HALF) return reinterpret_cast<const C*>(static_cast<const T*>(a.src) + base + 2 * (long long)e);
    return static_cast<const C*>(a.src) + base + (long long)e * a.in.es;
}

template <class C>
__device__ __forceinline__ void copy_async(unsigned d, const C* src)
{
    if constexpr (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void copy_async_wait()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Writes output elements e0, e0 + de, ... (< n_out) of one line, whose
// transform result sits in slots sl[k * LDB]; the op's post-processing is
// fixed at compile time and the global address advances as a running
// pointer.
template <int OP, bool BLUE, class C, class T>
__device__ __forceinline__ void store_elems(const StageArgs& a, const C* sl, int LDB, long long base, int e0, int de)
{
    const int n_out = a.n_out;
    const long long step = (long long)de * a.out.es;
    const C* chirp = static_cast<const C*>(a.chirp);
    // transform result for bin k (Bluestein: times the chirp, un-swapped)
    auto res = [&](int k) -> C {
        C v = sl[k * LDB];
        if constexpr (BLUE) v = mul(ldg(chirp + k), swp(v));
        return v;
    };
    if constexpr (OP == OP_R2C_HALF) {
        // F[k] = (Z[k] + conj Z[n-k]) / 2 - i exp(-2 pi i k / Nx) (Z[k] - conj Z[n-k]) / 2
        const int n = a.nfft;
        const C* tw2 = static_cast<const C*>(a.tw2);
        C* p = static_cast<C*>(a.dst) + base + e0 * a.out.es;
        for (int e = e0; e < n_out; e += de, p += step) {
            const C zk = res(e == n ? 0 : e);
            const C zm = cnj(res(e == 0 ? 0 : n - e));
            const C q = mul(ldg(tw2 + e), sub(zk, zm));
            *p = mk<C>((T)0.5 * (zk.x + zm.x + q.y), (T)0.5 * (zk.y + zm.y - q.x));
        }
    } else if constexpr (OP == OP_DCT1) {
        C* p = static_cast<C*>(a.dst) + base + e0 * a.out.es;
        for (int e = e0; e < n_out; e += de, p += step) *p = res(e);
    } else if constexpr (OP == OP_DST1) {
        // Y[e] = i Z[e + 1] (forward sign: Z[k] = -2i sum x_j sin(pi k (j+1)/(n+1)))
        C* p = static_cast<C*>(a.dst) + base + e0 * a.out.es;
        for (int e = e0; e < n_out; e += de, p += step) {
            const C z = res(e + 1);
            *p = mk<C>(-z.y, z.x);
        }
    } else if constexpr (OP == OP_C2R_HALF) {
        // f[2j] = Re z[j], f[2j+1] = Im z[j]: one complex-sized store per j
        C* p = reinterpret_cast<C*>(static_cast<T*>(a.dst) + base) + e0;
        for (int e = e0; e < n_out; e += de, p += de) *p = swp(res(e));
    } else {  // OP_C2C, OP_COPY
        const bool sw = a.sign > 0;
        C* p = static_cast<C*>(a.dst) + base + e0 * a.out.es;
        for (int e = e0; e < n_out; e += de, p += step) {
            const C v = res(e);
            *p = sw ? swp(v) : v;
        }
    }
}

template <bool BLUE, class C, class T>
__device__ __forceinline__ void store_line(const StageArgs& a, const C* sl, int LDB, long long base, int e0, int de)
{
    switch (a.op) {
    case OP_R2C_HALF: store_elems<OP_R2C_HALF, BLUE, C, T>(a, sl, LDB, base, e0, de); break;
    case OP_DCT1: store_elems<OP_DCT1, BLUE, C, T>(a, sl, LDB, base, e0, de); break;
    case OP_DST1: store_elems<OP_DST1, BLUE, C, T>(a, sl, LDB, base, e0, de); break;
    case OP_C2R_HALF: store_elems<OP_C2R_HALF, BLUE, C, T>(a, sl, LDB, base, e0, de); break;
    default: store_elems<OP_C2C, BLUE, C, T>(a, sl, LDB, base, e0, de); break;
    }
}

// Resident CTAs per SM the register allocation is sized for.  FP32: three
// 256-thread CTAs (85 registers).  Measured on 7-smooth grids (384^3 pair,
// 64-grid batch): 0.99 / 8.44 ms against 1.09 / 8.67 ms with four CTAs at 64
// registers (which spill) and 1.29 / 9.49 ms with two at 128 -- with the
// asynchronous tile loads the kernel needs registers more than a fourth CTA.
// FP64 stays at two: three CTAs spill several hundred bytes for a gain of
// about 2 %.
#ifndef P3_GEN_MINB
#define P3_GEN_MINB 3
#endif
#ifndef P3_GEN_MINB_F64
#define P3_GEN_MINB_F64 2
#endif
// One tile (lines tile * B .. tile * B + B - 1) of a generic stage, by all
// blockDim.x threads of the CTA (at least a.threads); smem_raw holds a.smem
// bytes.
template <typename T>
__device__ __forceinline__ void stage_tile(const StageArgs& a, long long tile, unsigned char* smem_raw)
{
    typedef typename Cx<T>::t C;
    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int B = a.B, LDB = a.LDB;
    const int lb = __ffs(B) - 1;  // B is a power of two: x / B = x >> lb
    const long long L0 = tile * B;
    const int nload = a.blue ? a.m : a.nfft;  // slots filled per line
    const int nfill = a.blue ? a.nfft : nload;  // slots taken from the input
    C* s0 = reinterpret_cast<C*>(smem_raw);
    C* s1 = s0 + (size_t)nload * LDB;  // second buffer of the ping-pong passes

    // ---- load: HBM -> shared memory ------------------------------------
    // Lines of the tile and the elements a thread takes: with lanes walking
    // elements, warp w takes lines w, w + nw, ... and lane e0 elements
    // e0, e0 + 32, ...; otherwise thread tid takes line tid mod B, elements
    // tid / B, tid / B + NT / B, ...
    const bool sw_in = a.sign > 0 && (a.op == OP_C2C || a.op == OP_COPY);  // inverse: swapped input
    if (direct_load(a)) {
        // every slot is a copy of one input value (nfill == nload).  The
        // inverse's real/imaginary swap is applied by the first pass (or,
        // without passes, below); the c2r input F[0..n] is copied as it is
        // (F[n] to the second buffer, unused until the first pass) and
        // pre-twiddled in shared memory below.
        const bool ef = a.in_elem_fast;
        const int l0 = ef ? tid >> 5 : tid & (B - 1), dl = ef ? NT >> 5 : B;
        const int e0 = ef ? tid & 31 : tid >> lb, de = ef ? 32 : NT >> lb;
        const long long gstep = (long long)de * (a.op == OP_R2C_HALF ? 1 : a.in.es);  // complex values
        const unsigned sstep = (unsigned)(de * LDB * (int)sizeof(C));
        // X rows stored one after another: the tile is one contiguous run
        // of its rows' complex values, which all threads walk together
        const int rowc = a.op == OP_C2R_HALF ? nload + 1 : nload;  // complex values per input row
        if (P3_GEN_FLAT && sizeof(T) == 4 && ef && (a.op == OP_R2C_HALF || a.op == OP_C2R_HALF) && a.in.per >= a.nlines &&
            a.in.lstride == (a.op == OP_R2C_HALF ? 2LL * nload : (long long)rowc)) {
            const long long rows = a.nlines - L0 < B ? a.nlines - L0 : B;
            const int total = (int)rows * rowc;
            const long long b0 = line_base(a.in, L0);
            const C* g0 = a.op == OP_R2C_HALF ? reinterpret_cast<const C*>(static_cast<const T*>(a.src) + b0)
                                              : static_cast<const C*>(a.src) + b0;
            int l = tid / rowc, e = tid - l * rowc;  // element i = l * rowc + e
            const int dq = NT / rowc, dr = NT - dq * rowc;
            for (int i = tid; i < total; i += NT) {
                copy_async((unsigned)__cvta_generic_to_shared(e < nload ? s0 + e * LDB + l : s1 + l), g0 + i);
                e += dr;
                l += dq;
                if (e >= rowc) {
                    e -= rowc;
                    ++l;
                }
            }
        } else {
            for (int l = l0; l < B; l += dl) {
                const long long L = L0 + l;
                if (L >= a.nlines) break;
                const long long base = line_base(a.in, L);
                const C* g = direct_src<C, T>(a, base, e0);
                unsigned sa = (unsigned)__cvta_generic_to_shared(s0 + e0 * LDB + l);
                for (int e = e0; e < nload; e += de) {
                    copy_async(sa, g);
                    g += gstep;
                    sa += sstep;
                }
                if (a.op == OP_C2R_HALF && e0 == 0)
                    copy_async((unsigned)__cvta_generic_to_shared(s1 + l), direct_src<C, T>(a, base, nload));
            }
        }
        copy_async_wait();
        if (sw_in && a.npass == 0) {
            for (int l = l0; l < B; l += dl) {
                if (L0 + l >= a.nlines) break;
                for (int e = e0; e < nload; e += de) s0[e * LDB + l] = swp(s0[e * LDB + l]);
            }
        }
        if (a.op == OP_C2R_HALF) {
            // Z[k] = (F[k] + conj F[n-k]) + i (F[k] - conj F[n-k]) exp(+2 pi i k / Nx)
            // (imaginary parts of F[0] and F[n] dropped), swapped for the
            // inverse FFT; the pair k, n - k is done by one thread, in place
            __syncthreads();
            const int n = a.nfft, half = n / 2 + 1;
            const C* tw2 = static_cast<const C*>(a.tw2);
            for (int i = tid; i < B * half; i += NT) {
                const int l = i & (B - 1), k = i >> lb;
                if (L0 + l >= a.nlines) continue;
                const int m = n - k;  // partner slot (F[n] for k = 0)
                C Fk = s0[(size_t)k * LDB + l];
                C Fm = k == 0 ? s1[l] : s0[(size_t)m * LDB + l];
                if (k == 0) {
                    Fk.y = (T)0;
                    Fm.y = (T)0;
                }
                {
                    const C B_ = cnj(Fm);
                    const C ze = add(Fk, B_);
                    const C zo = mul(sub(Fk, B_), cnj(ldg(tw2 + k)));
                    s0[(size_t)k * LDB + l] = swp(mk<C>(ze.x - zo.y, ze.y + zo.x));
                }
                if (k > 0 && m != k) {
                    const C B_ = cnj(Fk);
                    const C ze = add(Fm, B_);
                    const C zo = mul(sub(Fm, B_), cnj(ldg(tw2 + m)));
                    s0[(size_t)m * LDB + l] = swp(mk<C>(ze.x - zo.y, ze.y + zo.x));
                }
            }
        }
    } else {
        const bool ef = a.in_elem_fast;
        const int l0 = ef ? tid >> 5 : tid & (B - 1), dl = ef ? NT >> 5 : B;
        const int e0 = ef ? tid & 31 : tid >> lb, de = ef ? 32 : NT >> lb;
        const bool pair = a.op == OP_R2C_PAIR || a.op == OP_C2R_PAIR;
        for (int l = l0; l < B; l += dl) {
            const long long L = L0 + l;
            if (L >= a.nlines) break;
            if (pair) {
                const bool has2 = 2 * L + 1 < a.nrows;
                const long long b0 = line_base(a.in, 2 * L), b1 = has2 ? line_base(a.in, 2 * L + 1) : b0;
                if (a.op == OP_R2C_PAIR) {
                    if (a.blue) pair_load<OP_R2C_PAIR, true, C, T>(a, s0, LDB, l, b0, b1, has2, e0, de, nload, nfill);
                    else pair_load<OP_R2C_PAIR, false, C, T>(a, s0, LDB, l, b0, b1, has2, e0, de, nload, nfill);
                } else {
                    if (a.blue) pair_load<OP_C2R_PAIR, true, C, T>(a, s0, LDB, l, b0, b1, has2, e0, de, nload, nfill);
                    else pair_load<OP_C2R_PAIR, false, C, T>(a, s0, LDB, l, b0, b1, has2, e0, de, nload, nfill);
                }
                continue;
            }
            const long long base = line_base(a.in, L);
            if (a.blue)
                load_line<true, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill);
            else
                load_line<false, C, T>(a, s0, LDB, l, base, e0, de, nload, nfill);
        }
    }
    __syncthreads();

    // ---- FFT of every tile line in shared memory -----------------------
    C* s = s0;
    {
        const int l = tid & (B - 1);
        const int t = tid >> lb;
        const bool act = tid < B * a.tpl;
        if (!a.blue) {
            s = run_passes<C, T>(s0, s1, LDB, l, t, a.tpl, act, a.nfft, a.npass, a.rad, a.pc,
                                 static_cast<const C*>(a.tw), sw_in && direct_load(a));
        } else {
            // Bluestein: DFT_m, pointwise product with the filter spectrum,
            // inverse DFT_m as swp(DFT_m(swp(.))); the 1/m is folded into bhat.
            const C* twm = static_cast<const C*>(a.twm);
            C* x = run_passes<C, T>(s0, s1, LDB, l, t, a.tpl, act, a.m, a.mpass, a.mrad, a.mpc, twm);
            const C* bh = static_cast<const C*>(a.bhat);
            for (int i = tid; i < a.m * B; i += NT) {
                const int k = i >> lb, ll = i & (B - 1);
                x[k * LDB + ll] = swp(mul(x[k * LDB + ll], ldg(bh + k)));
            }
            __syncthreads();
            s = run_passes<C, T>(x, x == s0 ? s1 : s0, LDB, l, t, a.tpl, act, a.m, a.mpass, a.mrad, a.mpc, twm);
        }
    }

    // ---- store: shared memory -> HBM -----------------------------------
    // X rows stored one after another: all threads walk the tile's output
    // values together (R2C: H bins per row; C2R: n real pairs per row)
    if (P3_GEN_FLAT && sizeof(T) == 4 && a.out_elem_fast && !a.blue && (a.op == OP_R2C_HALF || a.op == OP_C2R_HALF) &&
        a.out.per >= a.nlines && a.out.lstride == (a.op == OP_R2C_HALF ? (long long)a.n_out : 2LL * a.n_out)) {
        const int rowo = a.n_out;
        const long long rows = a.nlines - L0 < B ? a.nlines - L0 : B;
        const int total = (int)rows * rowo;
        const long long b0 = line_base(a.out, L0);
        int l = tid / rowo, e = tid - l * rowo;  // element i = l * rowo + e
        const int dq = NT / rowo, dr = NT - dq * rowo;
        if (a.op == OP_R2C_HALF) {
            // F[k] = (Z[k] + conj Z[n-k]) / 2 - i exp(-2 pi i k / Nx) (Z[k] - conj Z[n-k]) / 2
            const int n = a.nfft;
            const C* tw2 = static_cast<const C*>(a.tw2);
            C* g0 = static_cast<C*>(a.dst) + b0;
            for (int i = tid; i < total; i += NT) {
                const C* sl = s + l;
                const C zk = sl[(e == n ? 0 : e) * LDB];
                const C zm = cnj(sl[(e == 0 ? 0 : n - e) * LDB]);
                const C q = mul(ldg(tw2 + e), sub(zk, zm));
                g0[i] = mk<C>((T)0.5 * (zk.x + zm.x + q.y), (T)0.5 * (zk.y + zm.y - q.x));
                e += dr;
                l += dq;
                if (e >= rowo) {
                    e -= rowo;
                    ++l;
                }
            }
        } else {
            // f[2j] = Re z[j], f[2j+1] = Im z[j]: one complex-sized store per j
            C* g0 = reinterpret_cast<C*>(static_cast<T*>(a.dst) + b0);
            for (int i = tid; i < total; i += NT) {
                g0[i] = swp(s[e * LDB + l]);
                e += dr;
                l += dq;
                if (e >= rowo) {
                    e -= rowo;
                    ++l;
                }
            }
        }
    } else {
        const bool ef = a.out_elem_fast;
        const int l0 = ef ? tid >> 5 : tid & (B - 1), dl = ef ? NT >> 5 : B;
        const int e0 = ef ? tid & 31 : tid >> lb, de = ef ? 32 : NT >> lb;
        const bool pair = a.op == OP_R2C_PAIR || a.op == OP_C2R_PAIR;
        for (int l = l0; l < B; l += dl) {
            const long long L = L0 + l;
            if (L >= a.nlines) break;
            if (pair) {
                const bool has2 = 2 * L + 1 < a.nrows;
                const long long b0 = line_base(a.out, 2 * L), b1 = has2 ? line_base(a.out, 2 * L + 1) : b0;
                if (a.op == OP_R2C_PAIR) {
                    if (a.blue) pair_store<OP_R2C_PAIR, true, C, T>(a, s + l, LDB, b0, b1, has2, e0, de);
                    else pair_store<OP_R2C_PAIR, false, C, T>(a, s + l, LDB, b0, b1, has2, e0, de);
                } else {
                    if (a.blue) pair_store<OP_C2R_PAIR, true, C, T>(a, s + l, LDB, b0, b1, has2, e0, de);
                    else pair_store<OP_C2R_PAIR, false, C, T>(a, s + l, LDB, b0, b1, has2, e0, de);
                }
                continue;
            }
            const long long base = line_base(a.out, L);
            if (a.blue)
                store_line<true, C, T>(a, s + l, LDB, base, e0, de);
            else
                store_line<false, C, T>(a, s + l, LDB, base, e0, de);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kGenThreads, (sizeof(T) == 4 ? P3_GEN_MINB : P3_GEN_MINB_F64))
    stage_kernel(const __grid_constant__ StageArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stage_tile<T>(a, blockIdx.x, smem_raw);
}

template <typename T>
cudaError_t launch_stage(const StageArgs& a0, cudaStream_t st)
{
    if (a0.nlines <= 0) return cudaSuccess;
    const long long grid = (a0.nlines + a0.B - 1) / a0.B;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    StageArgs a = a0;
    const long long nl = a.nrows > a.nlines ? a.nrows : a.nlines;  // pair ops index rows
    line_magic(a.in, nl);
    line_magic(a.out, nl);
    generic_consts(a);
    stage_kernel<T><<<(unsigned)grid, a.threads, a.smem, st>>>(a);
    return cudaGetLastError();
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Batched persistent launch: every CTA takes tickets in order; a ticket is a
// tile of one (plan, stage) task.  Thread 0 claims a CTA's next ticket while
// the current tile runs (a CTA holds at most one unstarted ticket, larger
// than its current one, so the smallest unfinished ticket can always
// proceed), finds its task in the compact scheduling array, and waits
// (bounded) until every tile of the plan's previous stage finished -- once
// per task, as a finished stage stays finished.  The task's arguments are
// copied to shared memory only when the task changes, with the call's
// buffers filled in.  A wait that gives up marks *err and skips the tile
// (the output of that call is invalid), still counting it as finished so no
// wait behind it hangs.
#ifndef P3_BATCH_MINB
#define P3_BATCH_MINB P3_GEN_MINB
#endif
__global__ void __launch_bounds__(kMaxThreads, P3_BATCH_MINB) batch_kernel(const __grid_constant__ BatchLaunch b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StageArgs sa;
    __shared__ long long s_tile;
    __shared__ int s_task, s_ok;
    const int tid = threadIdx.x;
    int cur = -1;      // task whose arguments sit in sa
    unsigned next = 0;  // thread 0: the claimed, unstarted ticket
    int met = -1;       // thread 0: task whose dependency was seen finished
    if (tid == 0) next = atomicAdd(b.ctr, 1u);
    for (;;) {
        if (tid == 0) {
            const unsigned tk = next;
            int task = -1, ok = 1;
            if (tk < b.total) {
                int lo = 0, hi = b.ntasks - 1;  // last task with first <= tk
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (b.meta[mid].first <= tk) lo = mid;
                    else hi = mid - 1;
                }
                task = lo;
                s_tile = (long long)(tk - b.meta[lo].first);
                next = atomicAdd(b.ctr, 1u);
                const int dep = b.meta[lo].dep;
                if (dep >= 0 && met != lo) {
                    const unsigned need = b.meta[dep].ntiles + b.extra;
                    unsigned it = 0;
                    while (ld_acquire_u32(b.ctr + 1 + dep) < need) {
                        if (++it > b.spin_limit || ld_acquire_u32(b.err) != 0) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                    if (ok) met = lo;
                    else atomicOr(b.err, 1u);
                }
            }
            s_task = task;
            s_ok = ok;
        }
        __syncthreads();
        const int task = s_task;
        if (task < 0) return;
        if (task != cur) {
            // the arguments after the tensor map (unused by the generic
            // kernel); thread 0 alone writes the buffer pointers
            constexpr int wb = (int)((offsetof(StageArgs, dst) + sizeof(void*)) / sizeof(int));
            constexpr int nw = (int)(sizeof(StageArgs) / sizeof(int));
            const int* srcw = reinterpret_cast<const int*>(&b.tasks[task].a);
            int* dstw = reinterpret_cast<int*>(&sa);
            for (int i = wb + tid; i < nw; i += blockDim.x) dstw[i] = srcw[i];
            if (tid == 0) {
                const BatchMeta& m = b.meta[task];
                sa.src = b.buf[m.plan][m.src];
                sa.dst = b.buf[m.plan][m.dst];
            }
            __syncthreads();
            cur = task;
        }
        if (s_ok) stage_tile<float>(sa, s_tile, smem_raw);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(b.ctr + 1 + task, 1u);
        }
    }
}

}  // namespace

int batch_grid(size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kMaxThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

cudaError_t batch_launch(const BatchLaunch& b, int grid, size_t smem, cudaStream_t s)
{
    if (b.total == 0) return cudaSuccess;
    const cudaError_t e = cudaMemsetAsync(b.ctr, 0, sizeof(unsigned) * (size_t)(1 + b.ntasks), s);
    if (e != cudaSuccess) return e;
    batch_kernel<<<grid, kMaxThreads, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_stage_f32(const StageArgs& a, cudaStream_t s)
{
    if (a.tc) return tc_launch(a, s);
    return a.kern != KIND_GENERIC ? pow2_launch(a, true, s) : launch_stage<float>(a, s);
}
cudaError_t launch_stage_f64(const StageArgs& a, cudaStream_t s)
{
    return a.kern != KIND_GENERIC ? pow2_launch(a, false, s) : launch_stage<double>(a, s);
}

cudaError_t prepare_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(stage_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    e = pow2_prepare();
    if (e != cudaSuccess) return e;
    return tc_prepare();
}

}  // namespace p3
