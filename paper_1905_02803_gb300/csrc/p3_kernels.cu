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
#include "p3_internal.h"

namespace p3 {
namespace {

template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };

template <class C> __device__ __forceinline__ C mk(decltype(C().x) x, decltype(C().x) y)
{
    C r;
    r.x = x;
    r.y = y;
    return r;
}
template <class C> __device__ __forceinline__ C add(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C sub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C mul(C a, C b)
{
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __device__ __forceinline__ C cnj(C a) { return mk<C>(a.x, -a.y); }
// (re, im) -> (im, re): conj(i * conj(a)).  swp(DFT(swp(x))) is the
// inverse-sign DFT, so one forward FFT code serves both directions.
template <class C> __device__ __forceinline__ C swp(C a) { return mk<C>(a.y, a.x); }
// -i * a
template <class C> __device__ __forceinline__ C mmi(C a) { return mk<C>(a.y, -a.x); }
template <class C, class T> __device__ __forceinline__ C scl(C a, T s) { return mk<C>(a.x * s, a.y * s); }
// a * (cr + i ci) with constant parts
template <class C, class T> __device__ __forceinline__ C rot(C a, T cr, T ci)
{
    return mk<C>(a.x * cr - a.y * ci, a.x * ci + a.y * cr);
}

template <class C> __device__ __forceinline__ C ldg(const C* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Forward DFT butterflies of size R on v[0..R), exp(-2 pi i n m / R), in place.
// ---------------------------------------------------------------------------
template <class C, class T>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3)
{
    C s02 = add(a0, a2), d02 = sub(a0, a2), s13 = add(a1, a3), d13 = mmi(sub(a1, a3));
    a0 = add(s02, s13);
    a2 = sub(s02, s13);
    a1 = add(d02, d13);
    a3 = sub(d02, d13);
}

template <class C, class T, int R> struct Dft;

template <class C, class T> struct Dft<C, T, 2> {
    static __device__ __forceinline__ void run(C* v)
    {
        C a = v[0];
        v[0] = add(a, v[1]);
        v[1] = sub(a, v[1]);
    }
};

template <class C, class T> struct Dft<C, T, 4> {
    static __device__ __forceinline__ void run(C* v) { dft4<C, T>(v[0], v[1], v[2], v[3]); }
};

template <class C, class T> struct Dft<C, T, 8> {
    static __device__ __forceinline__ void run(C* v)
    {
        const T h = (T)0.7071067811865476;  // sqrt(1/2)
        C u0 = add(v[0], v[4]), u1 = add(v[1], v[5]), u2 = add(v[2], v[6]), u3 = add(v[3], v[7]);
        C w0 = sub(v[0], v[4]), w1 = sub(v[1], v[5]), w2 = sub(v[2], v[6]), w3 = sub(v[3], v[7]);
        w1 = mk<C>(h * (w1.x + w1.y), h * (w1.y - w1.x));   // * exp(-i pi/4)
        w2 = mmi(w2);                                       // * exp(-i pi/2)
        w3 = mk<C>(h * (w3.y - w3.x), -h * (w3.x + w3.y));  // * exp(-3i pi/4)
        dft4<C, T>(u0, u1, u2, u3);
        dft4<C, T>(w0, w1, w2, w3);
        v[0] = u0; v[2] = u1; v[4] = u2; v[6] = u3;
        v[1] = w0; v[3] = w1; v[5] = w2; v[7] = w3;
    }
};

template <class C, class T> struct Dft<C, T, 16> {
    // 16 = 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddle exp(-2 pi i n2 k1/16),
    // DFT4 over n2; the result X[k1 + 4 k2] lands in slot 4 k1 + k2.
    static __device__ __forceinline__ void run(C* v)
    {
        const T c1 = (T)0.9238795325112867, s1 = (T)0.3826834323650898, h = (T)0.7071067811865476;
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4<C, T>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
        v[5] = rot(v[5], c1, -s1);    // n2=1,k1=1: W^1
        v[9] = rot(v[9], h, -h);      // n2=1,k1=2: W^2
        v[13] = rot(v[13], s1, -c1);  // n2=1,k1=3: W^3
        v[6] = rot(v[6], h, -h);      // n2=2,k1=1: W^2
        v[10] = mmi(v[10]);           // n2=2,k1=2: W^4
        v[14] = rot(v[14], -h, -h);   // n2=2,k1=3: W^6
        v[7] = rot(v[7], s1, -c1);    // n2=3,k1=1: W^3
        v[11] = rot(v[11], -h, -h);   // n2=3,k1=2: W^6
        v[15] = rot(v[15], -c1, s1);  // n2=3,k1=3: W^9
        // A[n2][k1] sits at v[n2 + 4 k1]; DFT4 over n2 for each k1
        C o[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
            dft4<C, T>(a0, a1, a2, a3);
            o[k1] = a0; o[k1 + 4] = a1; o[k1 + 8] = a2; o[k1 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
};

template <class C, class T> struct Dft<C, T, 3> {
    static __device__ __forceinline__ void run(C* v)
    {
        const T s3 = (T)0.8660254037844386;  // sqrt(3)/2
        C t = add(v[1], v[2]), d = sub(v[1], v[2]);
        C m = mk<C>(v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y);
        v[0] = add(v[0], t);
        v[1] = mk<C>(m.x + s3 * d.y, m.y - s3 * d.x);
        v[2] = mk<C>(m.x - s3 * d.y, m.y + s3 * d.x);
    }
};

// Odd prime R: pair a_j with a_{R-j}; cos / sin of 2 pi t / R by table.
template <class C, class T, int R> struct DftOdd {
    static __device__ __forceinline__ T cs(int t)
    {
        if (R == 5) {
            const double c[5] = {1.0, 0.30901699437494745, -0.8090169943749473, -0.8090169943749473,
                                 0.30901699437494745};
            return (T)c[t];
        } else {
            const double c[7] = {1.0, 0.6234898018587336, -0.22252093395631434, -0.900968867902419,
                                 -0.900968867902419, -0.22252093395631434, 0.6234898018587336};
            return (T)c[t];
        }
    }
    static __device__ __forceinline__ T sn(int t)
    {
        if (R == 5) {
            const double s[5] = {0.0, 0.9510565162951535, 0.5877852522924732, -0.5877852522924732,
                                 -0.9510565162951535};
            return (T)s[t];
        } else {
            const double s[7] = {0.0, 0.7818314824680298, 0.9749279121818236, 0.43388373911755823,
                                 -0.43388373911755823, -0.9749279121818236, -0.7818314824680298};
            return (T)s[t];
        }
    }
    static __device__ __forceinline__ void run(C* v)
    {
        constexpr int h = (R - 1) / 2;
        C p[h], q[h];
#pragma unroll
        for (int j = 1; j <= h; ++j) {
            p[j - 1] = add(v[j], v[R - j]);
            q[j - 1] = sub(v[j], v[R - j]);
        }
        C a0 = v[0];
        C y0 = a0;
#pragma unroll
        for (int j = 0; j < h; ++j) y0 = add(y0, p[j]);
#pragma unroll
        for (int m = 1; m <= h; ++m) {
            C re = a0, im = mk<C>((T)0, (T)0);
#pragma unroll
            for (int j = 1; j <= h; ++j) {
                const T c = cs((j * m) % R), s = sn((j * m) % R);
                re = mk<C>(re.x + c * p[j - 1].x, re.y + c * p[j - 1].y);
                im = mk<C>(im.x + s * q[j - 1].x, im.y + s * q[j - 1].y);
            }
            v[m] = mk<C>(re.x + im.y, re.y - im.x);      // re - i im
            v[R - m] = mk<C>(re.x - im.y, re.y + im.x);  // re + i im
        }
        v[0] = y0;
    }
};
template <class C, class T> struct Dft<C, T, 5> {
    static __device__ __forceinline__ void run(C* v) { DftOdd<C, T, 5>::run(v); }
};
template <class C, class T> struct Dft<C, T, 7> {
    static __device__ __forceinline__ void run(C* v) { DftOdd<C, T, 7>::run(v); }
};

// ---------------------------------------------------------------------------
// One Stockham (autosort, decimation in time) pass of radix R over n points
// of every tile line.  Butterfly j reads elements j + r n/R, multiplies by
// exp(-2 pi i (j mod Ns) r / (Ns R)), does a size-R DFT and writes
// (j / Ns) Ns R + (j mod Ns) + r Ns.  Thread t of a line takes butterflies
// t, t + tpl, ...; all reads finish (barrier) before any write.
// ---------------------------------------------------------------------------
template <class C, class T, int R>
__device__ __noinline__ void pass_r(C* s, int LDB, int l, int t, int tpl, bool act, int n, int Ns,
                                       const C* tw, int ts)
{
    constexpr int BM = kVmax / R;
    const int nb = n / R;
    const int span = n / (Ns * R);
    C v[BM][R];
#pragma unroll
    for (int b = 0; b < BM; ++b) {
        const int j = t + b * tpl;
        if (act && j < nb) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = s[(j + r * nb) * LDB + l];
            const int k = (j % Ns) * span;
            if (k) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = mul(v[b][r], ldg(tw + (size_t)(k * r) * ts));
            }
            Dft<C, T, R>::run(v[b]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BM; ++b) {
        const int j = t + b * tpl;
        if (act && j < nb) {
            const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
            for (int r = 0; r < R; ++r) s[(base + r * Ns) * LDB + l] = v[b][r];
        }
    }
    __syncthreads();
}

template <class C, class T>
__device__ __forceinline__ void run_passes(C* s, int LDB, int l, int t, int tpl, bool act, int n, int npass,
                                           const int* rad, const C* tw, int ts)
{
    int Ns = 1;
    for (int p = 0; p < npass; ++p) {
        const int R = rad[p];
        switch (R) {
        case 16: pass_r<C, T, 16>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        case 8: pass_r<C, T, 8>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        case 4: pass_r<C, T, 4>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        case 2: pass_r<C, T, 2>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        case 3: pass_r<C, T, 3>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        case 5: pass_r<C, T, 5>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        case 7: pass_r<C, T, 7>(s, LDB, l, t, tpl, act, n, Ns, tw, ts); break;
        default: break;
        }
        Ns *= R;
    }
}

__device__ __forceinline__ long long line_base(const LineMap& m, long long L)
{
    return (L / m.per) * m.gstride + (L % m.per) * m.lstride;
}

// Value placed in shared-memory slot e of a line before the FFT.
template <class C, class T>
__device__ __forceinline__ C load_value(const StageArgs& a, long long base, int e)
{
    const long long es = a.in.es;
    C v;
    switch (a.op) {
    case OP_R2C_HALF: {  // z[j] = f[2j] + i f[2j+1]; rows are contiguous
        const T* f = static_cast<const T*>(a.src);
        v = *reinterpret_cast<const C*>(f + base + 2 * (long long)e);
        break;
    }
    case OP_R2C_FULL: {
        const T* f = static_cast<const T*>(a.src);
        v = mk<C>(f[base + (long long)e * es], (T)0);
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
    case OP_C2R_FULL: {
        // weighted, zero-padded half spectrum: w_0 = 1, w_k = 2 (k < H), 0 above
        const C* F = static_cast<const C*>(a.src);
        if (e < a.n_in) {
            v = F[base + (long long)e * es];
            if (e) v = scl(v, (T)2);
        } else {
            v = mk<C>((T)0, (T)0);
        }
        v = swp(v);
        break;
    }
    case OP_DCT1: {  // even extension y[e] = x[e] (e <= M), x[2M - e] (e > M)
        const C* X = static_cast<const C*>(a.src);
        const int M = a.n_in - 1;
        const int src = e <= M ? e : 2 * M - e;
        v = X[base + (long long)src * es];
        break;
    }
    default: {  // OP_C2C, OP_COPY
        const C* X = static_cast<const C*>(a.src);
        v = X[base + (long long)e * es];
        if (a.sign > 0) v = swp(v);
        break;
    }
    }
    if (a.blue) v = mul(v, ldg(static_cast<const C*>(a.chirp) + e));
    return v;
}

// Transform result for bin k of the line whose slots start at sl (stride LDB).
template <class C>
__device__ __forceinline__ C result(const StageArgs& a, const C* sl, int LDB, int k)
{
    C v = sl[k * LDB];
    if (a.blue) v = mul(ldg(static_cast<const C*>(a.chirp) + k), swp(v));
    return v;
}

// Write output element e of a line.
template <class C, class T>
__device__ __forceinline__ void store_value(const StageArgs& a, const C* sl, int LDB, long long base, int e)
{
    const long long es = a.out.es;
    switch (a.op) {
    case OP_R2C_HALF: {
        // F[k] = (Z[k] + conj Z[n-k]) / 2 - i exp(-2 pi i k / Nx) (Z[k] - conj Z[n-k]) / 2
        const int n = a.nfft;
        const C zk = result(a, sl, LDB, e == n ? 0 : e);
        const C zm = cnj(result(a, sl, LDB, e == 0 ? 0 : n - e));
        const C p = mul(ldg(static_cast<const C*>(a.tw2) + e), sub(zk, zm));
        const C F = mk<C>((T)0.5 * (zk.x + zm.x + p.y), (T)0.5 * (zk.y + zm.y - p.x));
        static_cast<C*>(a.dst)[base + (long long)e * es] = F;
        break;
    }
    case OP_R2C_FULL:
    case OP_DCT1:
        static_cast<C*>(a.dst)[base + (long long)e * es] = result(a, sl, LDB, e);
        break;
    case OP_C2R_HALF: {  // f[2j] = Re z[j], f[2j+1] = Im z[j]
        const C z = swp(result(a, sl, LDB, e));
        *reinterpret_cast<C*>(static_cast<T*>(a.dst) + base + 2 * (long long)e) = z;
        break;
    }
    case OP_C2R_FULL: {
        const C z = swp(result(a, sl, LDB, e));
        static_cast<T*>(a.dst)[base + (long long)e * es] = z.x;
        break;
    }
    default: {  // OP_C2C, OP_COPY
        C v = result(a, sl, LDB, e);
        if (a.sign > 0) v = swp(v);
        static_cast<C*>(a.dst)[base + (long long)e * es] = v;
        break;
    }
    }
}

template <typename T>
__global__ void __launch_bounds__(kMaxThreads) stage_kernel(const __grid_constant__ StageArgs a)
{
    typedef typename Cx<T>::t C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);

    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int B = a.B, LDB = a.LDB;
    const long long L0 = (long long)blockIdx.x * B;
    const int nload = a.blue ? a.m : a.nfft;  // slots filled per line
    const int nfill = a.blue ? a.nfft : nload;  // slots taken from the input

    // ---- load: HBM -> shared memory ------------------------------------
    if (a.in_elem_fast) {
        const int lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
        for (int l = warp; l < B; l += nw) {
            const long long L = L0 + l;
            if (L >= a.nlines) break;
            const long long base = line_base(a.in, L);
            for (int e = lane; e < nload; e += 32)
                s[e * LDB + l] = e < nfill ? load_value<C, T>(a, base, e) : mk<C>((T)0, (T)0);
        }
    } else {
        const int l = tid & (B - 1);
        const long long L = L0 + l;
        if (L < a.nlines) {
            const long long base = line_base(a.in, L);
            for (int e = tid / B; e < nload; e += NT / B)
                s[e * LDB + l] = e < nfill ? load_value<C, T>(a, base, e) : mk<C>((T)0, (T)0);
        }
    }
    __syncthreads();

    // ---- FFT of every tile line in shared memory -----------------------
    {
        const int l = tid & (B - 1);
        const int t = tid / B;
        const bool act = tid < B * a.tpl;
        if (!a.blue) {
            run_passes<C, T>(s, LDB, l, t, a.tpl, act, a.nfft, a.npass, a.rad, static_cast<const C*>(a.tw),
                             a.twn / (a.nfft > 0 ? a.nfft : 1));
        } else {
            // Bluestein: DFT_m, pointwise product with the filter spectrum,
            // inverse DFT_m as swp(DFT_m(swp(.))); the 1/m is folded into bhat.
            const C* twm = static_cast<const C*>(a.twm);
            run_passes<C, T>(s, LDB, l, t, a.tpl, act, a.m, a.mpass, a.mrad, twm, 1);
            const C* bh = static_cast<const C*>(a.bhat);
            for (int i = tid; i < a.m * B; i += NT) {
                const int k = i / B, ll = i - k * B;
                s[k * LDB + ll] = swp(mul(s[k * LDB + ll], ldg(bh + k)));
            }
            __syncthreads();
            run_passes<C, T>(s, LDB, l, t, a.tpl, act, a.m, a.mpass, a.mrad, twm, 1);
        }
    }

    // ---- store: shared memory -> HBM -----------------------------------
    if (a.out_elem_fast) {
        const int lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
        for (int l = warp; l < B; l += nw) {
            const long long L = L0 + l;
            if (L >= a.nlines) break;
            const long long base = line_base(a.out, L);
            for (int e = lane; e < a.n_out; e += 32) store_value<C, T>(a, s + l, LDB, base, e);
        }
    } else {
        const int l = tid & (B - 1);
        const long long L = L0 + l;
        if (L < a.nlines) {
            const long long base = line_base(a.out, L);
            for (int e = tid / B; e < a.n_out; e += NT / B) store_value<C, T>(a, s + l, LDB, base, e);
        }
    }
}

template <typename T>
cudaError_t launch_stage(const StageArgs& a, cudaStream_t st)
{
    if (a.nlines <= 0) return cudaSuccess;
    const long long grid = (a.nlines + a.B - 1) / a.B;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    stage_kernel<T><<<(unsigned)grid, a.threads, a.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_f32(const StageArgs& a, cudaStream_t s) { return launch_stage<float>(a, s); }
cudaError_t launch_stage_f64(const StageArgs& a, cudaStream_t s) { return launch_stage<double>(a, s); }

cudaError_t prepare_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(stage_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace p3
