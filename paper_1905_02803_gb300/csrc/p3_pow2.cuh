// Specialised stage kernels for power-of-two line lengths (64 .. 4096): the
// hot path of the 3D transform (Sect. 2, Sect. 3.3 of the P3DFFT paper) with
// every pass, radix, index and direction known at compile time.
//
// Column kernels (Y and Z stages: lines whose neighbours are adjacent in
// memory, elements far apart).  Lanes walk B adjacent lines, so each global
// access of a line element is one coalesced B-wide run.  Each thread keeps E
// values of one line in registers (E = 16 or 32, one radix-E butterfly per
// pass); the first Stockham pass loads its butterfly inputs straight from
// HBM, the last pass stores straight to HBM, and shared memory is touched only
// for the exchanges between passes.  The Z stage that writes (or, inverse,
// reads) the STRIDE1 ZYX layout (Table 1) routes that side through shared
// memory with lanes along the line, 128 contiguous bytes per line per warp:
// the fused re-orientation that replaces the paper's COLUMN all-to-all and
// local transpose.
//
// Row kernels (X stage: contiguous lines).  Lanes walk the butterflies of one
// row; the real-to-complex split of an even-length line (a length Nx/2 complex
// FFT of (f[2j], f[2j+1]) plus the post-twiddle) and its inverse pre-twiddle
// are fused into the first / last pass.
//
// Shared-memory slots.  Columns: element e of tile line l lives at
// cpad(e) * B + (l ^ sw(e)) with cpad(e) = e + e/16 + e/32; the padding keeps
// the stride-E writes of the first pass and the unit-stride reads of later
// passes in distinct banks for the two line groups of a half-warp, and the
// XOR swizzle (ZYX kernels only) does the same for the element-contiguous
// phases.  Rows: row l at l * RP, element e at e + e/E.  Offsets that are
// multiples of 32 split off cpad exactly, so most slot addresses are a
// per-thread base plus an immediate.
#pragma once

#include "p3_dft.cuh"
#include "p3_internal.h"

namespace p3 {
namespace pw {

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// Radix plan of an N-point line with E values per thread: radix E while it
// divides, then one remainder pass.
template <int N, int E> struct P2 {
    static constexpr int LOGN = ilog2(N), LOGE = ilog2(E);
    static constexpr int NFULL = LOGN / LOGE;
    static constexpr int REM = 1 << (LOGN - NFULL * LOGE);
    static constexpr int NPASS = NFULL + (REM > 1 ? 1 : 0);
    static constexpr int TPL = N / E;
    __host__ __device__ static constexpr int radix(int p) { return p < NFULL ? E : REM; }
    __host__ __device__ static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
};

__device__ __forceinline__ int cpad(int e) { return e + (e >> 4) + (e >> 5); }
__host__ __device__ constexpr int cpad_c(int e) { return e + (e >> 4) + (e >> 5); }

// Pass P: butterfly b of thread t is j = t + b * TPL; it reads j + r N/R and
// writes (j / NS) NS R + j % NS + r NS.  Each index is split into a per-thread
// part u(t) and a compile-time part K(b, r) with alignment UA of u.
template <int N, int E, int P> struct PassIdx {
    typedef P2<N, E> PL;
    static constexpr int R = PL::radix(P), NS = PL::ns(P), BM = E / R, TPL = PL::TPL;
    static __device__ __forceinline__ int in_u(int t) { return t; }
    __host__ __device__ static constexpr int in_K(int b, int r) { return b * TPL + r * (N / R); }
    static constexpr int IN_UA = 1;
    // NS <= TPL: j % NS = t % NS and j / NS = t / NS + b TPL / NS; otherwise j < NS
    static constexpr bool OUT_SPLIT = NS <= TPL;
    static __device__ __forceinline__ int out_u(int t) { return OUT_SPLIT ? (t / NS) * NS * R + (t % NS) : t; }
    __host__ __device__ static constexpr int out_K(int b, int r) { return OUT_SPLIT ? b * TPL * R + r * NS : b * TPL + r * NS; }
    static constexpr int OUT_UA = (NS == 1) ? R : 1;
};

template <class T, int B, bool SWZ> struct ColSlot {
    static constexpr int SH = (sizeof(T) == 8 && B >= 8) ? 0 : 1;
    static constexpr int SWM = B << SH;  // swizzle period in elements
    static __device__ __forceinline__ int at(int e, int l)
    {
        return SWZ ? cpad(e) * B + (l ^ ((e >> SH) & (B - 1))) : cpad(e) * B + l;
    }
    // slot of element u + K (K a constant after unrolling, u aligned to UA):
    // per-thread base plus immediate whenever that is exact
    static __device__ __forceinline__ int at_k(int u, int l, int K, int UA)
    {
        const bool padsplit = (K % 32) == 0 || (UA % 32) == 0;
        if (!padsplit) return at(u + K, l);
        if (!SWZ || (K % SWM) == 0) return at(u, l) + cpad_c(K) * B;
        if ((UA % SWM) == 0) return cpad(u) * B + cpad_c(K) * B + (l ^ ((K >> SH) & (B - 1)));
        return at(u + K, l);
    }
};

template <class T> struct CxT;
template <> struct CxT<float> { typedef float2 t; };
template <> struct CxT<double> { typedef double2 t; };

#ifndef P3_E32_MINB
#define P3_E32_MINB 2
#endif
template <int NT, int CSIZE, int E> struct MinBlocks {
    static constexpr int value =
        CSIZE == 8 ? (E == 32 ? (NT >= 512 ? 1 : P3_E32_MINB) : (NT >= 512 ? 2 : 3)) : (NT >= 512 ? 1 : 2);
};

__device__ __forceinline__ long long lbase(const LineMap& m, long long L)
{
    if (m.pm) {  // L < 2^31: quotient by multiply-high (line_magic)
        const unsigned u = (unsigned)L;
        const unsigned q = (unsigned)(((unsigned long long)u * m.pm) >> m.ps);
        const unsigned r = u - q * (unsigned)m.per;
        return (long long)q * m.gstride + (long long)r * m.lstride;
    }
    return (L / m.per) * m.gstride + (L % m.per) * m.lstride;
}

// Line of lane l of tile `tile` (tile i takes lines i * B + l); false past
// the end.
__device__ __forceinline__ bool tile_line(const StageArgs& a, int B, long long tile, int l, long long* L)
{
    *L = tile * B + l;
    return *L < a.nlines;
}

// Cache policy of a tile's global loads / stores.  Loads: LD_CG through L2
// only (data another CTA of the same launch wrote: the SM's L1 may hold
// stale sectors of it); LD_CS streaming (read once, evict first).  Stores:
// ST_CS streaming (not read again soon).
enum { LD_DEF = 0, LD_CG = 1, LD_CS = 2 };
enum { ST_DEF = 0, ST_CS = 1 };
template <int LP, class C> __device__ __forceinline__ C ldx(const C* p)
{
    if constexpr (LP == LD_CG) return __ldcg(p);
    else if constexpr (LP == LD_CS) return __ldcs(p);
    else return *p;
}
template <int SP, class C> __device__ __forceinline__ void stx(C* p, const C& v)
{
    if constexpr (SP == ST_CS) __stcs(p, v);
    else *p = v;
}

// twiddle multiply of pass P for butterfly b (tw[k] = exp(-2 pi i k / twn),
// stride ts per FFT index), then DFT_R in registers
template <class C, class T, int N, int E, int P>
__device__ __forceinline__ void pass_compute(C (&v)[E], int t, const C* tw, int ts)
{
    typedef PassIdx<N, E, P> PI;
    constexpr int R = PI::R, NS = PI::NS;
#pragma unroll
    for (int b = 0; b < PI::BM; ++b) {
        if constexpr (NS > 1) {
            const int j = t + b * PI::TPL;
            const int step = (j % NS) * (N / (NS * R)) * ts;
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = mul(v[b * R + r], ldg(tw + step * r));
        }
        Dft<C, T, R>::run(&v[b * R]);
    }
}

// Row-twiddle tables: for lanes that run along a line (row-style kernels),
// the twiddles of pass P >= 1 are stored as entry (r - 1) NS + q, q = j % NS,
// so the lanes of a warp (consecutive j) read consecutive entries instead of
// entries j r apart.  Passes follow one another in one table.
template <int N, int E> __host__ __device__ constexpr int rtw_off(int P)
{
    return P <= 1 ? 0 : rtw_off<N, E>(P - 1) + (P2<N, E>::radix(P - 1) - 1) * P2<N, E>::ns(P - 1);
}

template <class C, class T, int N, int E, int P>
__device__ __forceinline__ void pass_compute_r(C (&v)[E], int t, const C* twr)
{
    typedef PassIdx<N, E, P> PI;
    constexpr int R = PI::R, NS = PI::NS, OFF = rtw_off<N, E>(P);
#pragma unroll
    for (int b = 0; b < PI::BM; ++b) {
        if constexpr (NS > 1) {
            const int q = (t + b * PI::TPL) % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = mul(v[b * R + r], ldg(twr + OFF + (r - 1) * NS + q));
        }
        Dft<C, T, R>::run(&v[b * R]);
    }
}

// Exchanges and passes 1 .. NP-1 through a column tile in shared memory.
template <class C, class T, int N, int E, int B, bool SWZ, int P, int NP> struct ColRest {
    static __device__ __forceinline__ void run(C (&v)[E], C* s, int l, int t, const C* tw)
    {
        typedef PassIdx<N, E, P - 1> Pr;
        typedef PassIdx<N, E, P> Cu;
        typedef ColSlot<T, B, SWZ> S;
        __syncthreads();
        {
            const int u = Pr::out_u(t);
#pragma unroll
            for (int b = 0; b < Pr::BM; ++b)
#pragma unroll
                for (int r = 0; r < Pr::R; ++r)
                    s[S::at_k(u, l, Pr::out_K(b, r), Pr::OUT_UA)] = v[b * Pr::R + r];
        }
        __syncthreads();
        {
            const int u = Cu::in_u(t);
#pragma unroll
            for (int b = 0; b < Cu::BM; ++b)
#pragma unroll
                for (int r = 0; r < Cu::R; ++r) v[b * Cu::R + r] = s[S::at_k(u, l, Cu::in_K(b, r), 1)];
        }
        pass_compute<C, T, N, E, P>(v, t, tw, 1);
        ColRest<C, T, N, E, B, SWZ, P + 1, NP>::run(v, s, l, t, tw);
    }
};
template <class C, class T, int N, int E, int B, bool SWZ, int NP> struct ColRest<C, T, N, E, B, SWZ, NP, NP> {
    static __device__ __forceinline__ void run(C (&)[E], C*, int, int, const C*) {}
};

template <class T, int N> __host__ __device__ constexpr int col_smem_slots() { return cpad_c(N - 1) + 1; }

// Element-contiguous phases of a column tile (the ZYX side): EL lanes per
// line, VEC elements per lane (16 bytes), 128 contiguous bytes of each of
// 32/EL lines per warp instruction.
template <class T, int N, int E, int B> struct EF {
    static constexpr int TPL = N / E, NT = B * TPL;
    static constexpr int VEC = sizeof(T) == 4 ? 2 : 1;
    static constexpr int ELD = sizeof(T) == 4 ? 16 : 8;
    static constexpr int EL = ELD < TPL ? ELD : TPL;
    static constexpr int STEP = NT / B;
    static __device__ __forceinline__ int line(int tid) { return (tid / EL) % B; }
    static __device__ __forceinline__ int chunk0(int tid) { return (tid % EL) + EL * (tid / (EL * B)); }
};

template <class T> struct Vec4;
template <> struct Vec4<float> { typedef float4 t; };

// MODE 0: HBM -> regs ... regs -> HBM (both sides line-adjacent)
// MODE 1: HBM -> regs ... smem -> HBM with lanes along elements (ZYX store)
// MODE 2: HBM (lanes along elements) -> smem -> regs ... regs -> HBM (ZYX load)
// INV: inverse sign (swp on load and store).
// SYM 0: plain line; 1: Chebyshev even extension (DCT-I of M + 1 points);
// 2: odd extension (DST-I of M - 1 points: element e reads 0 at e = 0, M,
// x[e - 1] below M and -x[N - 1 - e] above; output k is i times bin k + 1).
// One tile of B lines (tile index `tile`, lines offset by `off` elements in
// both arrays); s: the tile's shared memory.
template <typename T, int N, int E, int B, int MODE, bool INV, int SYM, int LP = LD_DEF, int SP = ST_DEF>
__device__ __forceinline__ void col_tile(const StageArgs& a, long long tile, long long off,
                                         typename CxT<T>::t* s)
{
    static_assert(SYM != 2 || !INV, "the sine transform always runs with the forward sign");
    constexpr bool DCT = SYM == 1, DST = SYM == 2;
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int NP = PL::NPASS;
    constexpr bool SWZ = MODE != 0;
    typedef ColSlot<T, B, SWZ> S;
    typedef EF<T, N, E, B> Ef;
    constexpr int M = N / 2;  // Chebyshev lines hold M + 1 points
    const int tid = threadIdx.x, l = tid % B, t = tid / B;
    long long L;
    const bool valid = tile_line(a, B, tile, l, &L);
    const C zero = mk<C>((T)0, (T)0);
    const C* tw = static_cast<const C*>(a.tw);
    C v[E];
    typedef PassIdx<N, E, 0> P0;

    if constexpr (MODE != 2) {
        const C* src = static_cast<const C*>(a.src) + off + (valid ? lbase(a.in, L) : 0);
        const long long es = a.in.es;
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) {
                const int K = P0::in_K(b, r);
                const int e = t + K;
                C x;
                if constexpr (DST) {
                    const long long o = (long long)(e < M ? e - 1 : N - 1 - e) * es;
                    x = (valid && e != 0 && e != M) ? ldx<LP>(src + o) : zero;
                    if (e > M) x = mk<C>(-x.x, -x.y);
                } else {
                    // even extension of a Chebyshev line: element e > M reads N - e
                    const long long o = DCT ? (long long)(e <= M ? e : N - e) * es : (long long)e * es;
                    x = valid ? ldx<LP>(src + o) : zero;
                }
                v[b * P0::R + r] = INV ? swp(x) : x;
            }
    } else {
        const int le = Ef::line(tid);
        long long Le;
        const bool ve = tile_line(a, B, tile, le, &Le);
        const C* src = static_cast<const C*>(a.src) + off + (ve ? lbase(a.in, Le) : 0);
        if constexpr (DST) {
            for (int c = Ef::chunk0(tid); c < N; c += Ef::STEP) {
                C x = (ve && c != 0 && c != M) ? ldx<LP>(src + (c < M ? c - 1 : N - 1 - c)) : zero;
                s[S::at(c, le)] = c > M ? mk<C>(-x.x, -x.y) : x;
            }
        } else if constexpr (DCT || Ef::VEC == 1) {
            for (int c = Ef::chunk0(tid); c < N; c += Ef::STEP) {
                const int ee = DCT ? (c <= M ? c : N - c) : c;
                C x = ve ? ldx<LP>(src + ee) : zero;
                s[S::at(c, le)] = INV ? swp(x) : x;
            }
        } else {
            typedef typename Vec4<T>::t V;
            const V* src4 = reinterpret_cast<const V*>(src);
            for (int c = Ef::chunk0(tid); c < N / 2; c += Ef::STEP) {
                V q = ve ? ldx<LP>(src4 + c) : V{(T)0, (T)0, (T)0, (T)0};
                C x0 = mk<C>(q.x, q.y), x1 = mk<C>(q.z, q.w);
                s[S::at(2 * c, le)] = INV ? swp(x0) : x0;
                s[S::at(2 * c + 1, le)] = INV ? swp(x1) : x1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) v[b * P0::R + r] = s[S::at(t + P0::in_K(b, r), l)];
    }
    pass_compute<C, T, N, E, 0>(v, t, tw, 1);
    ColRest<C, T, N, E, B, SWZ, 1, NP>::run(v, s, l, t, tw);

    typedef PassIdx<N, E, NP - 1> PLast;
    if constexpr (MODE != 1) {
        if (valid) {
            C* dst = static_cast<C*>(a.dst) + off + lbase(a.out, L);
            const long long es = a.out.es;
            const int u = PLast::out_u(t);
#pragma unroll
            for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
                for (int r = 0; r < PLast::R; ++r) {
                    const int e = u + PLast::out_K(b, r);
                    const C x = v[b * PLast::R + r];
                    if constexpr (DST) {
                        if (e >= 1 && e < M) stx<SP>(dst + (long long)(e - 1) * es, mk<C>(-x.y, x.x));
                    } else {
                        if (!DCT || e <= M) stx<SP>(dst + (long long)e * es, INV ? swp(x) : x);
                    }
                }
        }
    } else {
        __syncthreads();
        {
            const int u = PLast::out_u(t);
#pragma unroll
            for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
                for (int r = 0; r < PLast::R; ++r)
                    s[S::at_k(u, l, PLast::out_K(b, r), PLast::OUT_UA)] = v[b * PLast::R + r];
        }
        __syncthreads();
        const int le = Ef::line(tid);
        long long Le;
        if (tile_line(a, B, tile, le, &Le)) {
            C* dst = static_cast<C*>(a.dst) + off + lbase(a.out, Le);
            if constexpr (DST) {
                for (int c = Ef::chunk0(tid); c < M - 1; c += Ef::STEP) {
                    const C x = s[S::at(c + 1, le)];
                    dst[c] = mk<C>(-x.y, x.x);
                }
            } else if constexpr (DCT || Ef::VEC == 1) {
                for (int c = Ef::chunk0(tid); c < (DCT ? M + 1 : N); c += Ef::STEP) {
                    const C x = s[S::at(c, le)];
                    dst[c] = INV ? swp(x) : x;
                }
            } else {
                typedef typename Vec4<T>::t V;
                V* dst4 = reinterpret_cast<V*>(dst);
                for (int c = Ef::chunk0(tid); c < N / 2; c += Ef::STEP) {
                    C x0 = s[S::at(2 * c, le)], x1 = s[S::at(2 * c + 1, le)];
                    if (INV) {
                        x0 = swp(x0);
                        x1 = swp(x1);
                    }
                    dst4[c] = V{x0.x, x0.y, x1.x, x1.y};
                }
            }
        }
    }
}

template <typename T, int N, int E, int B, int MODE, bool INV, int SYM>
__global__ void __launch_bounds__(B * (N / E), (MinBlocks<B * (N / E), 2 * sizeof(T), E>::value))
    col_kernel(const __grid_constant__ StageArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    col_tile<T, N, E, B, MODE, INV, SYM>(a, blockIdx.x, 0, reinterpret_cast<typename CxT<T>::t*>(smem_raw));
}

// ---------------------------------------------------------------------------
// ZYX-store column kernel with a TMA-staged input tile (forward Z stage).
// The tile's B lines are adjacent in memory and their elements es apart, so
// the tile is a 2D box of the array (lines inner, elements outer): one thread
// arms an mbarrier with the tile's byte count and issues the tensor copies
// (boxes of B x 256 into a dense [e][l] tile); the CTA waits on the barrier
// (bounded), takes the first pass from shared memory and continues as the
// column kernel's ZYX-store form.  A wait that gives up sets bit 2 of
// *a.err, waits (bounded) for the copies in flight and leaves the tile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

constexpr int kTmaRows = 256;  // box height (elements of a line)

// Copy barrier of a tile: arrival count 1, or 2 in the test mode of
// StageArgs::wait_extra (one arrival never comes, so the wait runs out).
__device__ __forceinline__ void copy_bar_init(unsigned bar, int extra)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(extra ? 2 : 1) : "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Every thread waits (at most a.spin polls) for the tile's copies; true when
// all threads saw them land.  Otherwise bit 2 of *a.err is set, the missing
// test-mode arrival is supplied, and the CTA waits (again bounded) for the
// copies still in flight into its shared memory before the caller leaves.
__device__ __forceinline__ bool copy_bar_wait(const StageArgs& a, unsigned bar)
{
    int ok = 0;
    for (unsigned it = 0; it < a.spin; ++it)
        if (mbar_try_wait(bar, 0)) {
            ok = 1;
            break;
        }
    if (__syncthreads_and(ok)) return true;
    if (threadIdx.x == 0) {
        atomicOr(a.err, 2u);
        if (a.wait_extra) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
    }
    __syncthreads();
    for (unsigned it = 0; it < a.spin && !mbar_try_wait(bar, 0); ++it) {
    }
    return false;
}

template <int N, int SYM> __host__ __device__ constexpr int tma_rows()
{
    return SYM == 1 ? N / 2 + 1 : SYM == 2 ? N / 2 - 1 : N;
}
template <typename T, int N, int B, int SYM> __host__ __device__ constexpr size_t tma_tile_bytes()
{
    return (size_t)((tma_rows<N, SYM>() + kTmaRows - 1) / kTmaRows) * kTmaRows * B * 2 * sizeof(T);
}

template <typename T, int N, int E, int B, int SYM>
__global__ void __launch_bounds__(B * (N / E), (MinBlocks<B * (N / E), 2 * sizeof(T), E>::value))
    col_kernel_tma(const __grid_constant__ StageArgs a)
{
    static_assert(sizeof(T) == 4, "TMA tiles of 8-byte complex elements");
    constexpr bool DCT = SYM == 1, DST = SYM == 2;
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int NP = PL::NPASS;
    typedef ColSlot<T, B, true> S;
    typedef EF<T, N, E, B> Ef;
    constexpr int M = N / 2;
    constexpr int NBOX = (tma_rows<N, SYM>() + kTmaRows - 1) / kTmaRows;
    constexpr unsigned TX = (unsigned)tma_tile_bytes<T, N, B, SYM>();
    constexpr size_t SLOTS = (size_t)col_smem_slots<T, N>() * B * sizeof(C);
    constexpr size_t AREA = SLOTS > TX ? SLOTS : TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 128-byte aligned tile (the dynamic block is requested 128 + 16 bytes larger)
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    C* s = reinterpret_cast<C*>(base);
    const unsigned bar = smem_u32(base + AREA);
    const int tid = threadIdx.x, l = tid % B, t = tid / B;
    const long long L0 = (long long)blockIdx.x * B;
    if (tid == 0) copy_bar_init(bar, a.wait_extra);
    __syncthreads();
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(TX) : "memory");
#pragma unroll
        for (int k = 0; k < NBOX; ++k)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(smem_u32(s + (size_t)k * kTmaRows * B)),
                "l"(reinterpret_cast<unsigned long long>(&a.tmap)), "r"((int)L0), "r"(k * kTmaRows), "r"(bar)
                : "memory");
    }
    if (!copy_bar_wait(a, bar)) return;
    const C zero = mk<C>((T)0, (T)0);
    const C* tw = static_cast<const C*>(a.tw);
    C v[E];
    typedef PassIdx<N, E, 0> P0;
#pragma unroll
    for (int b = 0; b < P0::BM; ++b)
#pragma unroll
        for (int r = 0; r < P0::R; ++r) {
            const int e = t + P0::in_K(b, r);
            C x;
            if constexpr (DST) {
                x = (e != 0 && e != M) ? s[(e < M ? e - 1 : N - 1 - e) * B + l] : zero;
                if (e > M) x = mk<C>(-x.x, -x.y);
            } else {
                x = s[(DCT ? (e <= M ? e : N - e) : e) * B + l];
            }
            v[b * P0::R + r] = x;
        }
    pass_compute<C, T, N, E, 0>(v, t, tw, 1);
    ColRest<C, T, N, E, B, true, 1, NP>::run(v, s, l, t, tw);  // starts with a block barrier

    typedef PassIdx<N, E, NP - 1> PLast;
    __syncthreads();
    {
        const int u = PLast::out_u(t);
#pragma unroll
        for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
            for (int r = 0; r < PLast::R; ++r) s[S::at_k(u, l, PLast::out_K(b, r), PLast::OUT_UA)] = v[b * PLast::R + r];
    }
    __syncthreads();
    const int le = Ef::line(tid);
    const long long Le = L0 + le;
    if (Le < a.nlines) {
        C* dst = static_cast<C*>(a.dst) + lbase(a.out, Le);
        if constexpr (DST) {
            for (int c = Ef::chunk0(tid); c < M - 1; c += Ef::STEP) {
                const C x = s[S::at(c + 1, le)];
                dst[c] = mk<C>(-x.y, x.x);
            }
        } else if constexpr (DCT) {
            for (int c = Ef::chunk0(tid); c < M + 1; c += Ef::STEP) dst[c] = s[S::at(c, le)];
        } else {
            typedef typename Vec4<T>::t V;
            V* dst4 = reinterpret_cast<V*>(dst);
            for (int c = Ef::chunk0(tid); c < N / 2; c += Ef::STEP) {
                const C x0 = s[S::at(2 * c, le)], x1 = s[S::at(2 * c + 1, le)];
                dst4[c] = V{x0.x, x0.y, x1.x, x1.y};
            }
        }
    }
}

template <typename T, int N, int B> __host__ __device__ constexpr size_t col_tma_smem(int sym)
{
    typedef typename CxT<T>::t C;
    const size_t slots = (size_t)col_smem_slots<T, N>() * B * sizeof(C);
    const size_t tx = sym == 1 ? tma_tile_bytes<T, N, B, 1>() : sym == 2 ? tma_tile_bytes<T, N, B, 2>()
                                                                         : tma_tile_bytes<T, N, B, 0>();
    return (slots > tx ? slots : tx) + 128 + 16;
}

// ---------------------------------------------------------------------------
// Row kernels: X stage, Nx = 2N real points per row, H = N + 1 bins; row
// L starts at L * lstride of its array (real rows may be padded).
// OPR 0: r2c (forward), OPR 1: c2r (inverse).
// ---------------------------------------------------------------------------
template <int N, int E> struct RowSlot {
    static constexpr int RP = N + N / E + 1;  // odd pitch between rows
    static __device__ __forceinline__ int at(int e) { return e + e / E; }
    static __device__ __forceinline__ int at_k(int u, int K, int UA)
    {
        if ((K % E) == 0 || (UA % E) == 0) return at(u) + K + K / E;
        return at(u + K);
    }
};

// A row's TPL threads lie in one warp when TPL <= 32 (the B rows of a tile
// never share shared memory), so the row exchanges need only a warp
// barrier; longer rows span warps and use the block barrier.
template <int TPL> __device__ __forceinline__ void row_sync()
{
    if constexpr (TPL <= 32 && 32 % TPL == 0) __syncwarp();
    else __syncthreads();
}

template <class C, class T, int N, int E, int P, int NP, int TS = 2> struct RowRest {
    static __device__ __forceinline__ void run(C (&v)[E], C* s, int t, const C* tw)
    {
        typedef PassIdx<N, E, P - 1> Pr;
        typedef PassIdx<N, E, P> Cu;
        typedef RowSlot<N, E> S;
        row_sync<N / E>();
        {
            const int u = Pr::out_u(t);
#pragma unroll
            for (int b = 0; b < Pr::BM; ++b)
#pragma unroll
                for (int r = 0; r < Pr::R; ++r)
                    s[S::at_k(u, Pr::out_K(b, r), Pr::OUT_UA)] = v[b * Pr::R + r];
        }
        row_sync<N / E>();
#pragma unroll
        for (int b = 0; b < Cu::BM; ++b)
#pragma unroll
            for (int r = 0; r < Cu::R; ++r) v[b * Cu::R + r] = s[S::at_k(t, Cu::in_K(b, r), 1)];
        if constexpr (TS == 0) pass_compute_r<C, T, N, E, P>(v, t, tw);  // tw: row-twiddle table
        else pass_compute<C, T, N, E, P>(v, t, tw, TS);
        RowRest<C, T, N, E, P + 1, NP, TS>::run(v, s, t, tw);
    }
};
template <class C, class T, int N, int E, int NP, int TS> struct RowRest<C, T, N, E, NP, NP, TS> {
    static __device__ __forceinline__ void run(C (&)[E], C*, int, const C*) {}
};

// Rows L0 .. L0 + B - 1 (those below Lend) of a row stage; s: the tile's
// shared memory.
template <typename T, int N, int E, int B, int OPR, int LP = LD_DEF, int SP = ST_DEF>
__device__ __forceinline__ void row_tile(const StageArgs& a, long long L0, long long Lend, typename CxT<T>::t* s)
{
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS;
    typedef RowSlot<N, E> S;
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long L = L0 + l;
    const bool valid = L < Lend;
    const C zero = mk<C>((T)0, (T)0);
    const C* tw2 = static_cast<const C*>(a.tw2);  // exp(-2 pi i k / 2N), k < 2N
    C* srow = s + l * S::RP;
    C v[E];
    typedef PassIdx<N, E, 0> P0;
    typedef PassIdx<N, E, NP - 1> PLast;

    if constexpr (OPR == 0) {
        // z[j] = f[2j] + i f[2j+1]
        const C* src = reinterpret_cast<const C*>(static_cast<const T*>(a.src) + (valid ? L * a.in.lstride : 0));
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) v[b * P0::R + r] = valid ? ldx<LP>(src + t + P0::in_K(b, r)) : zero;
    } else {
        // Z[k] = (F[k] + conj F[N-k]) + i (F[k] - conj F[N-k]) exp(+2 pi i k / 2N),
        // imaginary parts of F[0] and F[N] dropped; inverse via swp
        const C* src = static_cast<const C*>(a.src) + (valid ? L * a.in.lstride : 0);
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) {
                const int k = t + P0::in_K(b, r);
                C A = valid ? ldx<LP>(src + k) : zero;
                C Bc = valid ? cnj(ldx<LP>(src + (N - k))) : zero;
                if (k == 0) {
                    A.y = (T)0;
                    Bc.y = (T)0;
                }
                const C ze = add(A, Bc);
                const C zo = mul(sub(A, Bc), cnj(ldg(tw2 + k)));
                v[b * P0::R + r] = swp(mk<C>(ze.x - zo.y, ze.y + zo.x));
            }
    }
    pass_compute<C, T, N, E, 0>(v, t, tw2, 2);
    RowRest<C, T, N, E, 1, NP, 0>::run(v, srow, t, static_cast<const C*>(a.twr));

    if constexpr (OPR == 0) {
        row_sync<N / E>();
        {
            const int u = PLast::out_u(t);
#pragma unroll
            for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
                for (int r = 0; r < PLast::R; ++r)
                    srow[S::at_k(u, PLast::out_K(b, r), PLast::OUT_UA)] = v[b * PLast::R + r];
        }
        row_sync<N / E>();
        if (valid) {
            C* dst = static_cast<C*>(a.dst) + L * a.out.lstride;
            for (int k = t; k <= N; k += TPL) {
                const C zk = srow[S::at(k == N ? 0 : k)];
                const C zm = cnj(srow[S::at(k == 0 ? 0 : N - k)]);
                const C p = mul(ldg(tw2 + k), sub(zk, zm));
                stx<SP>(dst + k, mk<C>((T)0.5 * (zk.x + zm.x + p.y), (T)0.5 * (zk.y + zm.y - p.x)));
            }
        }
    } else {
        if (valid) {
            C* dst = reinterpret_cast<C*>(static_cast<T*>(a.dst) + L * a.out.lstride);
            const int u = PLast::out_u(t);
#pragma unroll
            for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
                for (int r = 0; r < PLast::R; ++r) stx<SP>(dst + u + PLast::out_K(b, r), swp(v[b * PLast::R + r]));
        }
    }
}

template <typename T, int N, int E, int B, int OPR>
__global__ void __launch_bounds__(B * (N / E), (MinBlocks<B * (N / E), 2 * sizeof(T), E>::value))
    row_kernel(const __grid_constant__ StageArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    row_tile<T, N, E, B, OPR>(a, (long long)blockIdx.x * B, a.nlines,
                              reinterpret_cast<typename CxT<T>::t*>(smem_raw));
}

// ---------------------------------------------------------------------------
// ZYX-load kernel with row-style lines (the inverse Z stage reading the
// STRIDE1 layout of Table 1).  Each input line is contiguous there, so a
// line's TPL threads load it like an X row (coalesced, straight into
// registers) and run the passes with exchanges private to the line's warp;
// the results cross shared memory once, to be stored with lanes across the
// tile's B adjacent lines (B-wide runs of the XYZ output).  Input lines must
// have unit element stride.  SYM as in col_tile.
// ---------------------------------------------------------------------------
template <typename T, int N, int E, int B> __host__ __device__ constexpr size_t zrow_area()
{
    typedef typename CxT<T>::t C;
    const size_t ex = (size_t)B * (size_t)RowSlot<N, E>::RP, res = (size_t)N * (size_t)B;
    return (ex > res ? ex : res) * sizeof(C);
}

// BULK: the tile's B lines are consecutive in memory (plain FFT lines), so
// one bulk copy brings them into shared memory against an mbarrier (bounded
// wait, as in col_kernel_tma) and the first pass reads them from there.
template <typename T, int N, int E, int B, bool INV, int SYM, bool BULK = false>
__global__ void __launch_bounds__(B * (N / E), (MinBlocks<B * (N / E), 2 * sizeof(T), E>::value))
    zrow_kernel(const __grid_constant__ StageArgs a)
{
    static_assert(SYM != 2 || !INV, "the sine transform always runs with the forward sign");
    static_assert(!BULK || SYM == 0, "bulk tiles of whole, even-length lines");
    constexpr bool DCT = SYM == 1, DST = SYM == 2;
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS, NT = B * TPL;
    constexpr int M = N / 2;
    // result tile: element e of line l at e * B + (l ^ sw(e)); the swizzle
    // spreads a warp's writes (one line, consecutive e) and keeps the store
    // phase's reads (B lines of consecutive e) on distinct banks
    constexpr int SWS = B >= 16 ? 0 : B == 8 ? 1 : 2;
    static_assert(NT % B == 0 && B >= 4, "store lanes keep their line");
    typedef RowSlot<N, E> S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = BULK ? smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u) : smem_raw;
    C* s = reinterpret_cast<C*>(base);
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long L0 = (long long)blockIdx.x * B;
    const long long L = L0 + l;
    const bool valid = L < a.nlines;
    const C zero = mk<C>((T)0, (T)0);
    const C* tw = static_cast<const C*>(a.tw);
    C v[E];
    typedef PassIdx<N, E, 0> P0;
    typedef PassIdx<N, E, NP - 1> PLast;
    if constexpr (BULK) {
        const unsigned bar = smem_u32(base + zrow_area<T, N, E, B>());
        const long long left = a.nlines - L0;
        const unsigned bytes = (unsigned)((left < B ? left : B) * N * (long long)sizeof(C));
        if (tid == 0) copy_bar_init(bar, a.wait_extra);
        __syncthreads();
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                             smem_u32(s)),
                         "l"(static_cast<const C*>(a.src) + lbase(a.in, L0)), "r"(bytes), "r"(bar)
                         : "memory");
        }
        if (!copy_bar_wait(a, bar)) return;
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) {
                const C x = valid ? s[l * N + t + P0::in_K(b, r)] : zero;
                v[b * P0::R + r] = INV ? swp(x) : x;
            }
        __syncthreads();  // the exchange rows overlap the bulk tile
    } else {
        const C* src = static_cast<const C*>(a.src) + (valid ? lbase(a.in, L) : 0);
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) {
                const int e = t + P0::in_K(b, r);
                C x;
                if constexpr (DST) {
                    x = (valid && e != 0 && e != M) ? src[e < M ? e - 1 : N - 1 - e] : zero;
                    if (e > M) x = mk<C>(-x.x, -x.y);
                } else {
                    x = valid ? src[DCT ? (e <= M ? e : N - e) : e] : zero;
                }
                v[b * P0::R + r] = INV ? swp(x) : x;
            }
    }
    pass_compute<C, T, N, E, 0>(v, t, tw, 1);
    RowRest<C, T, N, E, 1, NP, 0>::run(v, s + l * S::RP, t, static_cast<const C*>(a.twr));
    __syncthreads();  // the result tile overlaps other lines' exchange rows
    {
        const int u = PLast::out_u(t);
#pragma unroll
        for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
            for (int r = 0; r < PLast::R; ++r) {
                const int e = u + PLast::out_K(b, r);
                s[e * B + (l ^ ((e >> SWS) & (B - 1)))] = v[b * PLast::R + r];
            }
    }
    __syncthreads();
    constexpr int NOUT = DCT ? M + 1 : DST ? M - 1 : N;
    const int ll = tid % B;
    const long long LL = L0 + ll;
    if (LL < a.nlines) {
        C* dst = static_cast<C*>(a.dst) + lbase(a.out, LL);
        const long long es = a.out.es;
        for (int c = tid / B; c < NOUT; c += NT / B) {
            const int e = DST ? c + 1 : c;
            C x = s[e * B + (ll ^ ((e >> SWS) & (B - 1)))];
            if constexpr (DST) x = mk<C>(-x.y, x.x);
            else if constexpr (INV) x = swp(x);
            dst[(long long)c * es] = x;
        }
    }
}

template <typename T, int N, int E, int B> __host__ __device__ constexpr size_t zrow_smem()
{
    return zrow_area<T, N, E, B>();
}
template <typename T, int N, int E, int B> __host__ __device__ constexpr size_t zrow_bulk_smem()
{
    return zrow_area<T, N, E, B>() + 128 + 16;
}

// ---------------------------------------------------------------------------
// Tile shapes per precision and length
// ---------------------------------------------------------------------------
#ifndef P3_COL_E32
#define P3_COL_E32 1
#endif
// E = 32 (two radix-32 passes for 1024 points) for the FP32 kernels whose
// first pass reads HBM directly; the ZYX-load kernel keeps E = 16.
template <typename T> __host__ __device__ constexpr int col_E(int N, int mode)
{
    return (sizeof(T) == 4 && P3_COL_E32 && mode != 2 && N >= 512 && N <= 2048) ? 32 : 16;
}
template <typename T> __host__ __device__ constexpr int col_B(int N)
{
    return sizeof(T) == 4 ? (N <= 64 ? 64 : N <= 128 ? 32 : N <= 256 ? 16 : N <= 2048 ? 8 : 4)
                          : (N <= 64 ? 64 : N <= 128 ? 32 : N <= 256 ? 16 : N <= 512 ? 8 : N <= 2048 ? 4 : 2);
}

// Row-style ZYX-load kernel for FP32 lines of 256 .. 2048 points (a line's
// threads fit in one warp up to 1024 points; two warps at 2048).
#ifndef P3_ZROW
#define P3_ZROW 1
#endif
template <typename T> __host__ __device__ constexpr bool col_zrow(int N)
{
    return P3_ZROW && sizeof(T) == 4 && N >= 256 && N <= 2048;
}
#ifndef P3_ROW_E32
#define P3_ROW_E32 1
#endif
// Row kernels: E = 32 (two passes for 512 / 1024 half-length points) for
// FP32 rows of 512 .. 2048, else 16; B rows so that a CTA has 256 threads.
template <typename T> __host__ __device__ constexpr int row_E(int N)
{
    return (sizeof(T) == 4 && P3_ROW_E32 && N >= 512 && N <= 2048) ? 32 : 16;
}
template <typename T> __host__ __device__ constexpr int row_B(int N)
{
    return (256 / (N / row_E<T>(N))) > 0 ? 256 / (N / row_E<T>(N)) : 1;
}
// lines per tile of the row-style ZYX-load kernel: a CTA of 256 threads, or
// 8 lines (512 threads) at 2048 points so the strided stores keep 64-byte runs
template <typename T> __host__ __device__ constexpr int zrow_B(int N) { return N >= 2048 ? 8 : row_B<T>(N); }

}  // namespace pw
}  // namespace p3
