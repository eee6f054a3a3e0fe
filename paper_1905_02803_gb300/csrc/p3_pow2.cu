// Specialised stage kernels for power-of-two line lengths (64 .. 4096): the
// hot path of the 3D transform (Sect. 2, Sect. 3.3 of the P3DFFT paper) with
// every pass, radix and index known at compile time.
//
// Column kernels (Y and Z stages: lines whose neighbours are adjacent in
// memory, elements far apart).  Lanes walk B adjacent lines, so each global
// access of a line element is one coalesced B-wide run.  Each thread keeps
// E = 16 values of one line in registers; the first Stockham pass loads its
// butterfly inputs straight from HBM, the last pass stores straight to HBM,
// and shared memory is touched only for the exchanges between passes.  The
// Z stage that writes (or, inverse, reads) the STRIDE1 ZYX layout (Table 1)
// routes that side through shared memory so that the transposed HBM access
// still moves whole 32-byte sectors: this is the fused re-orientation that
// replaces the paper's COLUMN all-to-all and local transpose.
//
// Row kernels (X stage: contiguous lines).  Lanes walk the butterflies of one
// row; the real-to-complex split of an even-length line (a length Nx/2
// complex FFT of (f[2j], f[2j+1]) plus the post-twiddle) and its inverse
// pre-twiddle are fused into the first / last pass.
//
// Shared memory holds element e of line l at (e + e/16) * B + l (columns) or
// l * RP + e + e/16 (rows): the spare slot every 16 elements keeps the
// stride-16 writes of a radix-16 pass free of bank conflicts.
#include "p3_dft.cuh"
#include "p3_internal.h"

namespace p3 {
namespace {

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

constexpr int kE = 16;  // values per thread

template <int N> struct P2 {
    static constexpr int LOGN = ilog2(N), LOGE = ilog2(kE);
    static constexpr int NFULL = LOGN / LOGE;
    static constexpr int REM = 1 << (LOGN - NFULL * LOGE);
    static constexpr int NPASS = NFULL + (REM > 1 ? 1 : 0);
    static constexpr int TPL = N / kE;
    static constexpr int radix(int p) { return p < NFULL ? kE : REM; }
    static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
};

__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

__device__ __forceinline__ long long lbase(const LineMap& m, long long L)
{
    return (L / m.per) * m.gstride + (L % m.per) * m.lstride;
}

// Pass P of the Stockham FFT over N points: butterfly b of thread t is
// j = t + b * TPL; it reads j + r N/R and writes (j/NS) NS R + j%NS + r NS.
template <class C, class T, int N, int P> struct Pass {
    typedef P2<N> PL;
    static constexpr int R = PL::radix(P), NS = PL::ns(P), BM = kE / R, TPL = PL::TPL;
    static __device__ __forceinline__ int in_idx(int t, int b, int r) { return t + b * TPL + r * (N / R); }
    static __device__ __forceinline__ int out_idx(int t, int b, int r)
    {
        const int j = t + b * TPL;
        return (j / NS) * NS * R + (j % NS) + r * NS;
    }
    // twiddle exp(-2 pi i (j%NS) r / (NS R)) = tw[((j%NS) r N/(NS R)) ts], then DFT_R
    static __device__ __forceinline__ void compute(C (&v)[kE], int t, const C* tw, int ts)
    {
#pragma unroll
        for (int b = 0; b < BM; ++b) {
            if (NS > 1) {
                const int j = t + b * TPL;
                const int k = (j % NS) * (N / (NS * R)) * ts;
#pragma unroll
                for (int r = 1; r < R; ++r) v[b * R + r] = mul(v[b * R + r], ldg(tw + k * r));
            }
            Dft<C, T, R>::run(&v[b * R]);
        }
    }
};

// Passes P .. NPASS-1 for a shared-memory line view sl(e) = s[idx(e)].
template <class C, class T, int N, int P, int NP> struct Rest {
    template <class Idx>
    static __device__ __forceinline__ void run(C (&v)[kE], C* s, Idx idx, int t, const C* tw, int ts)
    {
        typedef Pass<C, T, N, P - 1> Prev;
        typedef Pass<C, T, N, P> Cur;
        __syncthreads();
#pragma unroll
        for (int b = 0; b < Prev::BM; ++b)
#pragma unroll
            for (int r = 0; r < Prev::R; ++r) s[idx(Prev::out_idx(t, b, r))] = v[b * Prev::R + r];
        __syncthreads();
#pragma unroll
        for (int b = 0; b < Cur::BM; ++b)
#pragma unroll
            for (int r = 0; r < Cur::R; ++r) v[b * Cur::R + r] = s[idx(Cur::in_idx(t, b, r))];
        Cur::compute(v, t, tw, ts);
        Rest<C, T, N, P + 1, NP>::run(v, s, idx, t, tw, ts);
    }
};
template <class C, class T, int N, int NP> struct Rest<C, T, N, NP, NP> {
    template <class Idx>
    static __device__ __forceinline__ void run(C (&)[kE], C*, Idx, int, const C*, int)
    {
    }
};

template <class T> struct CxT;
template <> struct CxT<float> { typedef float2 t; };
template <> struct CxT<double> { typedef double2 t; };

template <int NT, int CSIZE> struct MinBlocks {
    static constexpr int value = CSIZE == 8 ? (NT >= 512 ? 2 : 3) : (NT >= 512 ? 1 : 2);
};

// MODE 0: HBM -> regs ... regs -> HBM (both sides line-adjacent)
// MODE 1: HBM -> regs ... smem -> HBM with lanes along elements (ZYX store)
// MODE 2: HBM (lanes along elements) -> smem -> regs ... regs -> HBM (ZYX load)
template <typename T, int N, int B, int MODE>
__global__ void __launch_bounds__(B * (N / kE), (MinBlocks<B * (N / kE), 2 * sizeof(T)>::value))
    col_kernel(const __grid_constant__ StageArgs a)
{
    typedef typename CxT<T>::t C;
    typedef P2<N> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, l = tid % B, t = tid / B;
    const long long L = (long long)blockIdx.x * B + l;
    const bool valid = L < a.nlines;
    const bool inv = a.sign > 0;
    const bool dct = a.op == OP_DCT1;
    constexpr int M = N / 2;  // Chebyshev lines hold M + 1 points
    const C zero = mk<C>((T)0, (T)0);
    const C* tw = static_cast<const C*>(a.tw);
    auto sidx = [l](int e) { return pad16(e) * B + l; };
    C v[kE];
    typedef Pass<C, T, N, 0> P0;

    if (MODE != 2) {
        const C* src = static_cast<const C*>(a.src) + (valid ? lbase(a.in, L) : 0);
        const long long es = a.in.es;
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) {
                const int e = P0::in_idx(t, b, r);
                const int ee = dct ? (e <= M ? e : N - e) : e;
                C x = valid ? src[ee * es] : zero;
                v[b * P0::R + r] = inv ? swp(x) : x;
            }
    } else {
        const C* src = static_cast<const C*>(a.src) + (valid ? lbase(a.in, L) : 0);
        for (int e = t; e < N; e += TPL) {
            const int ee = dct ? (e <= M ? e : N - e) : e;
            C x = valid ? src[ee] : zero;
            s[sidx(e)] = inv ? swp(x) : x;
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) v[b * P0::R + r] = s[sidx(P0::in_idx(t, b, r))];
    }
    P0::compute(v, t, tw, 1);
    Rest<C, T, N, 1, NP>::run(v, s, sidx, t, tw, 1);

    typedef Pass<C, T, N, NP - 1> PLast;
    const int nout = dct ? M + 1 : N;
    if (MODE != 1) {
        if (valid) {
            C* dst = static_cast<C*>(a.dst) + lbase(a.out, L);
            const long long es = a.out.es;
#pragma unroll
            for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
                for (int r = 0; r < PLast::R; ++r) {
                    const int e = PLast::out_idx(t, b, r);
                    const C x = v[b * PLast::R + r];
                    if (!dct || e <= M) dst[e * es] = inv ? swp(x) : x;
                }
        }
    } else {
        __syncthreads();
#pragma unroll
        for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
            for (int r = 0; r < PLast::R; ++r) s[sidx(PLast::out_idx(t, b, r))] = v[b * PLast::R + r];
        __syncthreads();
        if (valid) {
            C* dst = static_cast<C*>(a.dst) + lbase(a.out, L);
            for (int e = t; e < nout; e += TPL) {
                const C x = s[sidx(e)];
                dst[e] = inv ? swp(x) : x;
            }
        }
    }
}

// Row kernels: X stage, Nx = 2N real points per row, H = N + 1 bins.
// OPR 0: r2c (forward), OPR 1: c2r (inverse).
template <typename T, int N, int B, int OPR>
__global__ void __launch_bounds__(B * (N / kE), (MinBlocks<B * (N / kE), 2 * sizeof(T)>::value))
    row_kernel(const __grid_constant__ StageArgs a)
{
    typedef typename CxT<T>::t C;
    typedef P2<N> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS;
    constexpr int RP = N + N / 16 + 1;  // row pitch in slots
    constexpr int H = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long L = (long long)blockIdx.x * B + l;
    const bool valid = L < a.nlines;
    const C zero = mk<C>((T)0, (T)0);
    const C* tw2 = static_cast<const C*>(a.tw2);  // exp(-2 pi i k / 2N), k < 2N
    C* srow = s + l * RP;
    auto sidx = [](int e) { return pad16(e); };
    C v[kE];
    typedef Pass<C, T, N, 0> P0;
    typedef Pass<C, T, N, NP - 1> PLast;

    if (OPR == 0) {
        // z[j] = f[2j] + i f[2j+1]
        const C* src = reinterpret_cast<const C*>(static_cast<const T*>(a.src) + (valid ? L * (2LL * N) : 0));
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) v[b * P0::R + r] = valid ? src[P0::in_idx(t, b, r)] : zero;
    } else {
        // Z[k] = (F[k] + conj F[N-k]) + i (F[k] - conj F[N-k]) exp(+2 pi i k / 2N),
        // imaginary parts of F[0] and F[N] dropped; inverse via swp
        const C* src = static_cast<const C*>(a.src) + (valid ? L * (long long)H : 0);
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) {
                const int k = P0::in_idx(t, b, r);
                C A = valid ? src[k] : zero;
                C Bc = valid ? cnj(src[N - k]) : zero;
                if (k == 0) {
                    A.y = (T)0;
                    Bc.y = (T)0;
                }
                const C ze = add(A, Bc);
                const C zo = mul(sub(A, Bc), cnj(ldg(tw2 + k)));
                v[b * P0::R + r] = swp(mk<C>(ze.x - zo.y, ze.y + zo.x));
            }
    }
    P0::compute(v, t, tw2, 2);
    Rest<C, T, N, 1, NP>::run(v, srow, sidx, t, tw2, 2);

    if (OPR == 0) {
        __syncthreads();
#pragma unroll
        for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
            for (int r = 0; r < PLast::R; ++r) srow[sidx(PLast::out_idx(t, b, r))] = v[b * PLast::R + r];
        __syncthreads();
        if (valid) {
            C* dst = static_cast<C*>(a.dst) + L * (long long)H;
            for (int k = t; k <= N; k += TPL) {
                const C zk = srow[sidx(k == N ? 0 : k)];
                const C zm = cnj(srow[sidx(k == 0 ? 0 : N - k)]);
                const C p = mul(ldg(tw2 + k), sub(zk, zm));
                dst[k] = mk<C>((T)0.5 * (zk.x + zm.x + p.y), (T)0.5 * (zk.y + zm.y - p.x));
            }
        }
    } else {
        if (valid) {
            C* dst = reinterpret_cast<C*>(static_cast<T*>(a.dst) + L * (2LL * N));
#pragma unroll
            for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
                for (int r = 0; r < PLast::R; ++r) dst[PLast::out_idx(t, b, r)] = swp(v[b * PLast::R + r]);
        }
    }
}

// ---------------------------------------------------------------------------
// Configuration and dispatch
// ---------------------------------------------------------------------------
template <typename T> constexpr int col_B(int N)
{
    return sizeof(T) == 4 ? (N <= 64 ? 64 : N <= 128 ? 32 : N <= 256 ? 16 : N <= 1024 ? 8 : N <= 2048 ? 4 : 2)
                          : (N <= 64 ? 64 : N <= 128 ? 32 : N <= 256 ? 16 : N <= 512 ? 8 : N <= 2048 ? 4 : 2);
}
template <typename T> constexpr int row_B(int N) { return N <= 64 ? 64 : N <= 128 ? 32 : N <= 256 ? 16 : N <= 512 ? 8 : N <= 1024 ? 4 : N <= 2048 ? 2 : 1; }

template <typename T, int N, int MODE> void* col_fn() { return (void*)col_kernel<T, N, col_B<T>(N), MODE>; }
template <typename T, int N, int OPR> void* row_fn() { return (void*)row_kernel<T, N, row_B<T>(N), OPR>; }

template <typename T> void* pick(int kind, int N)
{
#define P3_COLS(NN)                                              \
    case NN:                                                     \
        switch (kind) {                                          \
        case KIND_COL_DD: return col_fn<T, NN, 0>();             \
        case KIND_COL_DS: return col_fn<T, NN, 1>();             \
        case KIND_COL_SD: return col_fn<T, NN, 2>();             \
        case KIND_ROW_R2C: return row_fn<T, NN, 0>();            \
        case KIND_ROW_C2R: return row_fn<T, NN, 1>();            \
        default: return nullptr;                                 \
        }
    switch (N) {
        P3_COLS(64)
        P3_COLS(128)
        P3_COLS(256)
        P3_COLS(512)
        P3_COLS(1024)
        P3_COLS(2048)
        P3_COLS(4096)
    default: return nullptr;
    }
#undef P3_COLS
}

bool is_pow2_in_range(int n) { return n >= 64 && n <= 4096 && (n & (n - 1)) == 0; }

}  // namespace

bool pow2_configure(StageArgs& a, size_t csize)
{
    if (a.blue) return false;
    const int N = a.nfft;
    if (!is_pow2_in_range(N)) return false;
    const bool f32 = csize == 8;
    int kind = 0;
    if (a.op == OP_C2C || a.op == OP_DCT1) {
        const bool in_adj = a.in.lstride == 1, out_adj = a.out.lstride == 1;
        const bool in_el = a.in.es == 1, out_el = a.out.es == 1;
        if (in_adj && out_adj && !in_el && !out_el) kind = KIND_COL_DD;
        else if (in_adj && !in_el && out_el) kind = KIND_COL_DS;
        else if (in_el && out_adj && !out_el) kind = KIND_COL_SD;
        else return false;
        const int B = f32 ? col_B<float>(N) : col_B<double>(N);
        a.B = B;
        a.LDB = B;
        a.tpl = N / kE;
        a.threads = B * a.tpl;
        a.smem = (size_t)(N + N / 16) * B * csize;
    } else if (a.op == OP_R2C_HALF || a.op == OP_C2R_HALF) {
        if (a.in.es != 1 || a.out.es != 1) return false;
        kind = a.op == OP_R2C_HALF ? KIND_ROW_R2C : KIND_ROW_C2R;
        const int B = f32 ? row_B<float>(N) : row_B<double>(N);
        a.B = B;
        a.LDB = N + N / 16 + 1;
        a.tpl = N / kE;
        a.threads = B * a.tpl;
        a.smem = (size_t)B * (N + N / 16 + 1) * csize;
    } else {
        return false;
    }
    a.kern = kind;
    return true;
}

cudaError_t pow2_prepare()
{
    for (int f = 0; f < 2; ++f)
        for (int kind = KIND_COL_DD; kind <= KIND_ROW_C2R; ++kind)
            for (int N = 64; N <= 4096; N *= 2) {
                void* fn = f == 0 ? pick<float>(kind, N) : pick<double>(kind, N);
                if (!fn) continue;
                cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

cudaError_t pow2_launch(const StageArgs& a, bool f32, cudaStream_t st)
{
    void* fn = f32 ? pick<float>(a.kern, a.nfft) : pick<double>(a.kern, a.nfft);
    if (!fn) return cudaErrorInvalidDeviceFunction;
    if (a.nlines <= 0) return cudaSuccess;
    const long long grid = (a.nlines + a.B - 1) / a.B;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    void* args[] = {const_cast<StageArgs*>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(a.threads), args, a.smem, st);
}

}  // namespace p3
