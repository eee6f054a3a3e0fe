// Tensor-core split-precision column kernels (FP32 data, 1024-point lines):
// the Y and Z stages of the 3D transform (Sect. 2 of the P3DFFT paper) with
// their two radix-16 Stockham passes done as dense products on the tensor
// cores, the final radix-4 pass on the CUDA cores.
//
// A radix-16 pass applies the 16-point DFT to every butterfly column: with
// C[m][r] = cos(2 pi m r / 16) and S[m][r] = sin(2 pi m r / 16),
//   Re y = C xr + S xi,   Im y = C xi - S xr.
// Each 16 x 16 real product runs as m16n8k8 TF32 MMAs over an n-tile of 8
// columns (one butterfly of the tile's 8 lines).  To keep FP32 accuracy every
// FP32 operand is split into a TF32 head and a TF32 tail (x = hi + lo, lo the
// rounding remainder) and the product is hi*hi + hi*lo + lo*hi, accumulated in
// FP32; TF32 keeps FP32's exponent range, so no per-tile scaling is needed.
//
// Tile: 8 adjacent lines, 512 threads (16 warps); warp w owns butterflies
// w, w + 16, w + 32, w + 48 of both radix-16 passes.  Loads, stores, the ZYX
// element-contiguous phases and the shared-memory slots are those of the
// FP32 1024-point column kernels (p3_pow2.cuh).
#include <stdint.h>

#include "p3_pow2.cuh"

namespace p3 {
namespace tcs {

using namespace pw;

constexpr int N = 1024, B = 8, TPL = 64, NT = B * TPL;

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragments of C and S (heads and tails) for k-tiles 0 and 1.  Lane
// (g, q) = (lane / 4, lane % 4) holds rows g, g + 8 and columns q, q + 4 of
// each 16 x 8 block.
struct WFrag {
    uint32_t ch[2][4], cl[2][4], sh[2][4], sl[2][4];
};

__device__ __forceinline__ void load_w(WFrag& w, int lane)
{
    // cos / sin(2 pi t / 16), t = 0..15
    const double c16[16] = {1.0, 0.9238795325112867, 0.7071067811865476, 0.3826834323650898, 0.0,
                            -0.3826834323650898, -0.7071067811865476, -0.9238795325112867, -1.0,
                            -0.9238795325112867, -0.7071067811865476, -0.3826834323650898, 0.0,
                            0.3826834323650898, 0.7071067811865476, 0.9238795325112867};
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
        const int rows[4] = {g, g + 8, g, g + 8};
        const int cols[4] = {kt * 8 + q, kt * 8 + q, kt * 8 + q + 4, kt * 8 + q + 4};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int t = (rows[i] * cols[i]) & 15;
            const float c = (float)c16[t];
            const float s = (float)c16[(t + 12) & 15];  // sin(a) = cos(a - pi/2)
            split(c, w.ch[kt][i], w.cl[kt][i]);
            split(s, w.sh[kt][i], w.sl[kt][i]);
        }
    }
}

// 16-point DFT of the 8 columns of one n-tile.  x: this lane's inputs of
// line g at r = q, q + 4, q + 8, q + 12.  y: outputs (m, line) =
// (g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1).
__device__ __forceinline__ void dft16_tc(const WFrag& w, const float2 (&x)[4], float2 (&y)[4])
{
    uint32_t rh[4], rl[4], ih[4], il[4], nrh[4], nrl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        split(x[i].x, rh[i], rl[i]);
        split(x[i].y, ih[i], il[i]);
        nrh[i] = rh[i] ^ 0x80000000u;  // -xr, exact sign flip
        nrl[i] = rl[i] ^ 0x80000000u;
    }
    // four independent accumulator chains (C xr, S xi, C xi, -S xr) so that
    // consecutive MMAs do not wait on each other
    float ra[4] = {0.f, 0.f, 0.f, 0.f}, rb[4] = {0.f, 0.f, 0.f, 0.f};
    float ia[4] = {0.f, 0.f, 0.f, 0.f}, ib[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
        const int b0 = 2 * kt, b1 = 2 * kt + 1;  // x[b0] is r = 8kt + q, x[b1] is r = 8kt + q + 4
        mma(ra, w.ch[kt], rh[b0], rh[b1]);
        mma(rb, w.sh[kt], ih[b0], ih[b1]);
        mma(ia, w.ch[kt], ih[b0], ih[b1]);
        mma(ib, w.sh[kt], nrh[b0], nrh[b1]);
        mma(ra, w.ch[kt], rl[b0], rl[b1]);
        mma(rb, w.sh[kt], il[b0], il[b1]);
        mma(ia, w.ch[kt], il[b0], il[b1]);
        mma(ib, w.sh[kt], nrl[b0], nrl[b1]);
        mma(ra, w.cl[kt], rh[b0], rh[b1]);
        mma(rb, w.sl[kt], ih[b0], ih[b1]);
        mma(ia, w.cl[kt], ih[b0], ih[b1]);
        mma(ib, w.sl[kt], nrh[b0], nrh[b1]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) y[i] = make_float2(ra[i] + rb[i], ia[i] + ib[i]);
}

// MODE as in col_kernel: 0 strided in/out, 1 ZYX store, 2 ZYX load.
template <int MODE, bool INV>
__global__ void __launch_bounds__(NT, 1) col_tc_kernel(const __grid_constant__ StageArgs a)
{
    typedef float2 C;
    constexpr bool SWZ = MODE != 0;
    typedef ColSlot<float, B, SWZ> S;
    typedef EF<float, N, 16, B> Ef;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, q = lane & 3;
    const C zero = make_float2(0.f, 0.f);
    const C* tw = static_cast<const C*>(a.tw);  // exp(-2 pi i k / 1024)
    WFrag w;
    load_w(w, lane);

    // ---- pass 0 inputs: butterfly j reads elements j + 64 r ------------
    C xin[4][4];
    {
        const long long Lg = (long long)blockIdx.x * B + g;  // this lane's line in the B operand
        const bool vg = Lg < a.nlines;
        if constexpr (MODE != 2) {
            const C* src = static_cast<const C*>(a.src) + (vg ? lbase(a.in, Lg) : 0);
            const long long es = a.in.es;
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = warp + 16 * n, r = q + 4 * i;
                    C x = vg ? src[(long long)(j + 64 * r) * es] : zero;
                    xin[n][i] = INV ? swp(x) : x;
                }
        } else {
            const int le = Ef::line(tid);
            long long Le = (long long)blockIdx.x * B + le;
            const bool ve = Le < a.nlines;
            const C* src = static_cast<const C*>(a.src) + (ve ? lbase(a.in, Le) : 0);
            const float4* src4 = reinterpret_cast<const float4*>(src);
            for (int c = Ef::chunk0(tid); c < N / 2; c += Ef::STEP) {
                float4 v = ve ? src4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                C x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
                s[S::at(2 * c, le)] = INV ? swp(x0) : x0;
                s[S::at(2 * c + 1, le)] = INV ? swp(x1) : x1;
            }
            __syncthreads();
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int i = 0; i < 4; ++i) xin[n][i] = s[S::at(warp + 16 * n + 64 * (q + 4 * i), g)];
            __syncthreads();
        }
    }
    // ---- pass 0 (radix 16, Ns = 1): outputs at 16 j + m ----------------
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const int j = warp + 16 * n;
        C y[4];
        dft16_tc(w, xin[n], y);
        s[S::at(16 * j + g, 2 * q)] = y[0];
        s[S::at(16 * j + g, 2 * q + 1)] = y[1];
        s[S::at(16 * j + g + 8, 2 * q)] = y[2];
        s[S::at(16 * j + g + 8, 2 * q + 1)] = y[3];
    }
    __syncthreads();
    // ---- pass 1 (radix 16, Ns = 16): twiddle exp(-2 pi i (j%16) r 4/1024) --
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = warp + 16 * n, r = q + 4 * i;
            C x = s[S::at(j + 64 * r, g)];
            const int k = (j & 15) * 4 * r;
            if (k) x = mul(x, ldg(tw + k));
            xin[n][i] = x;
        }
    __syncthreads();
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const int j = warp + 16 * n;
        const int ob = (j >> 4) * 256 + (j & 15);
        C y[4];
        dft16_tc(w, xin[n], y);
        s[S::at(ob + 16 * g, 2 * q)] = y[0];
        s[S::at(ob + 16 * g, 2 * q + 1)] = y[1];
        s[S::at(ob + 16 * (g + 8), 2 * q)] = y[2];
        s[S::at(ob + 16 * (g + 8), 2 * q + 1)] = y[3];
    }
    __syncthreads();
    // ---- pass 2 (radix 4, Ns = 256) on the CUDA cores -------------------
    const int l = tid % B, t = tid / B;
    const long long L = (long long)blockIdx.x * B + l;
    const bool valid = L < a.nlines;
    C v[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = t + 64 * b;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            C x = s[S::at(j + 256 * r, l)];
            if (r) x = mul(x, ldg(tw + j * r));
            v[4 * b + r] = x;
        }
        Dft<C, float, 4>::run(&v[4 * b]);
    }
    if constexpr (MODE != 1) {
        if (valid) {
            C* dst = static_cast<C*>(a.dst) + lbase(a.out, L);
            const long long es = a.out.es;
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const C x = v[4 * b + r];
                    dst[(long long)(t + 64 * b + 256 * r) * es] = INV ? swp(x) : x;
                }
        }
    } else {
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int r = 0; r < 4; ++r) s[S::at(t + 64 * b + 256 * r, l)] = v[4 * b + r];
        __syncthreads();
        const int le = Ef::line(tid);
        const long long Le = (long long)blockIdx.x * B + le;
        if (Le < a.nlines) {
            C* dst = static_cast<C*>(a.dst) + lbase(a.out, Le);
            float4* dst4 = reinterpret_cast<float4*>(dst);
            for (int c = Ef::chunk0(tid); c < N / 2; c += Ef::STEP) {
                C x0 = s[S::at(2 * c, le)], x1 = s[S::at(2 * c + 1, le)];
                if (INV) {
                    x0 = swp(x0);
                    x1 = swp(x1);
                }
                dst4[c] = make_float4(x0.x, x0.y, x1.x, x1.y);
            }
        }
    }
}

void* pick(int kind, bool inv)
{
    switch (kind) {
    case KIND_COL_DD: return inv ? (void*)col_tc_kernel<0, true> : (void*)col_tc_kernel<0, false>;
    case KIND_COL_DS: return inv ? (void*)col_tc_kernel<1, true> : (void*)col_tc_kernel<1, false>;
    case KIND_COL_SD: return inv ? (void*)col_tc_kernel<2, true> : (void*)col_tc_kernel<2, false>;
    default: return nullptr;
    }
}

}  // namespace tcs

// Configure a stage for the tensor-core split kernels (FP32, 1024-point C2C
// column stages); false when they do not apply.
bool tc_configure(StageArgs& a, size_t csize)
{
    if (csize != 8 || a.op != OP_C2C || a.nfft != tcs::N || a.blue) return false;
    if (a.kern != KIND_COL_DD && a.kern != KIND_COL_DS && a.kern != KIND_COL_SD) return false;
    a.B = tcs::B;
    a.LDB = tcs::B;
    a.tpl = tcs::TPL;
    a.threads = tcs::NT;
    a.smem = (size_t)(pw::cpad_c(tcs::N - 1) + 1) * tcs::B * csize;
    a.tc = 1;
    return true;
}

cudaError_t tc_prepare()
{
    for (int kind = KIND_COL_DD; kind <= KIND_COL_SD; ++kind)
        for (int inv = 0; inv < 2; ++inv) {
            cudaError_t e = cudaFuncSetAttribute(tcs::pick(kind, inv), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 227 * 1024);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t tc_launch(const StageArgs& a, cudaStream_t st)
{
    void* fn = tcs::pick(a.kern, a.sign > 0);
    if (!fn) return cudaErrorInvalidDeviceFunction;
    if (a.nlines <= 0) return cudaSuccess;
    const long long grid = (a.nlines + a.B - 1) / a.B;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    void* args[] = {const_cast<StageArgs*>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(a.threads), args, a.smem, st);
}

}  // namespace p3
