// Complex helpers and forward DFT butterflies (exp(-2 pi i n m / R)) of
// sizes 2, 3, 4, 5, 7, 8, 16 and 32 on registers, and of the composite sizes
// 6 .. 28 built from them, shared by the stage kernels.
// The inverse-sign DFT is swp(DFT(swp(x))), so only the forward form exists.
#pragma once

#include <cuda_runtime.h>

namespace p3 {

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

// FP32 complex add / subtract as one packed two-lane instruction
// (add.rn.f32x2 / sub.rn.f32x2, sm_100 and later): the same two IEEE
// round-to-nearest operations, in half the issue slots.
__device__ __forceinline__ unsigned long long pk2(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ float2 sub(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
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
// a + (-i) t and a - (-i) t (lanes swap, so no packed form)
template <class C> __device__ __forceinline__ C add_mmi(C a, C t) { return mk<C>(a.x + t.y, a.y - t.x); }
template <class C> __device__ __forceinline__ C sub_mmi(C a, C t) { return mk<C>(a.x - t.y, a.y + t.x); }
// a times exp(-i pi / 4) and exp(-3 i pi / 4): two adds and one scale
template <class C, class T> __device__ __forceinline__ C rot45(C a)
{
    const T h = (T)0.7071067811865476;
    return mk<C>(h * (a.x + a.y), h * (a.y - a.x));
}
template <class C, class T> __device__ __forceinline__ C rot135(C a)
{
    const T h = (T)0.7071067811865476;
    return mk<C>(h * (a.y - a.x), -h * (a.x + a.y));
}

// DFT4; with R2 the true a2 is -i times the given one (a rotation folded in)
template <class C, class T, bool R2 = false>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3)
{
    const C s02 = R2 ? add_mmi(a0, a2) : add(a0, a2), d02 = R2 ? sub_mmi(a0, a2) : sub(a0, a2);
    const C s13 = add(a1, a3), t = sub(a1, a3);
    a0 = add(s02, s13);
    a2 = sub(s02, s13);
    a1 = add_mmi(d02, t);
    a3 = sub_mmi(d02, t);
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
        C u0 = add(v[0], v[4]), u1 = add(v[1], v[5]), u2 = add(v[2], v[6]), u3 = add(v[3], v[7]);
        C w0 = sub(v[0], v[4]), w1 = sub(v[1], v[5]), w2 = sub(v[2], v[6]), w3 = sub(v[3], v[7]);
        w1 = rot45<C, T>(w1);   // * exp(-i pi/4)
        w3 = rot135<C, T>(w3);  // * exp(-3i pi/4)
        dft4<C, T>(u0, u1, u2, u3);
        dft4<C, T, true>(w0, w1, w2, w3);  // w2 * exp(-i pi/2) folded in
        v[0] = u0; v[2] = u1; v[4] = u2; v[6] = u3;
        v[1] = w0; v[3] = w1; v[5] = w2; v[7] = w3;
    }
};

template <class C, class T> struct Dft<C, T, 16> {
    // 16 = 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddle exp(-2 pi i n2 k1/16),
    // DFT4 over n2; the result X[k1 + 4 k2] lands in slot 4 k1 + k2.  With
    // R8 the true v[8] is -i times the given one.
    template <bool R8 = false> static __device__ __forceinline__ void run(C* v)
    {
        const T c1 = (T)0.9238795325112867, s1 = (T)0.3826834323650898;
        dft4<C, T, R8>(v[0], v[4], v[8], v[12]);
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2) dft4<C, T>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
        v[5] = rot(v[5], c1, -s1);    // n2=1,k1=1: W^1
        v[9] = rot45<C, T>(v[9]);     // n2=1,k1=2: W^2
        v[13] = rot(v[13], s1, -c1);  // n2=1,k1=3: W^3
        v[6] = rot45<C, T>(v[6]);     // n2=2,k1=1: W^2
        // n2=2,k1=2: W^4 = -i, folded into the k1 = 2 DFT4 below
        v[14] = rot135<C, T>(v[14]);  // n2=2,k1=3: W^6
        v[7] = rot(v[7], s1, -c1);    // n2=3,k1=1: W^3
        v[11] = rot135<C, T>(v[11]);  // n2=3,k1=2: W^6
        v[15] = rot(v[15], -c1, s1);  // n2=3,k1=3: W^9
        // A[n2][k1] sits at v[n2 + 4 k1]; DFT4 over n2 for each k1
        C o[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
            if (k1 == 2)
                dft4<C, T, true>(a0, a1, a2, a3);
            else
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
// 32 = 2 x 16 (decimation in frequency): u_k = a_k + a_{k+16},
// w_k = (a_k - a_{k+16}) exp(-2 pi i k / 32); even bins DFT16(u), odd DFT16(w).
template <class C, class T> struct Dft<C, T, 32> {
    static __device__ __forceinline__ void run(C* v)
    {
        // cos(pi k / 16), k = 0..8; sin(pi k / 16) = cos(pi (8 - k) / 16)
        const T c[9] = {(T)1.0, (T)0.9807852804032304, (T)0.9238795325112867, (T)0.8314696123025452,
                        (T)0.7071067811865476, (T)0.5555702330196022, (T)0.3826834323650898,
                        (T)0.19509032201612825, (T)0.0};
        C u[16], w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            u[k] = add(v[k], v[k + 16]);
            const C d = sub(v[k], v[k + 16]);
            // angle pi k / 16: cos / sin from the first-octant table; k = 0
            // is 1, k = 8 is -i (folded into DFT16's first DFT4), k = 4 and
            // 12 are the 45 and 135 degree rotations
            const T ck = k <= 8 ? c[k] : -c[16 - k];
            const T sk = k <= 8 ? c[8 - k] : c[k - 8];
            w[k] = k == 0 || k == 8 ? d : k == 4 ? rot45<C, T>(d) : k == 12 ? rot135<C, T>(d) : rot(d, ck, -sk);
        }
        Dft<C, T, 16>::run(u);
        Dft<C, T, 16>::template run<true>(w);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[2 * k] = u[k];
            v[2 * k + 1] = w[k];
        }
    }
};

template <class C, class T> struct Dft<C, T, 5> {
    static __device__ __forceinline__ void run(C* v) { DftOdd<C, T, 5>::run(v); }
};
template <class C, class T> struct Dft<C, T, 7> {
    static __device__ __forceinline__ void run(C* v) { DftOdd<C, T, 7>::run(v); }
};

// ---------------------------------------------------------------------------
// Compile-time cos / sin of 2 pi m / n (the composite butterflies' internal
// twiddles): the angle is reduced to the first octant, where the Taylor
// series of sin and cos converge to double precision within 13 terms
// (x <= pi/4: x^26 / 26! < 1e-28).
// ---------------------------------------------------------------------------
struct KTrigVal {
    double c, s;
};
__host__ __device__ constexpr KTrigVal ksincos_octant(double x)  // 0 <= x <= pi/4
{
    double c = 0.0, s = 0.0, tc = 1.0, ts = x;
    for (int k = 0; k < 13; ++k) {
        c += tc;
        s += ts;
        tc *= -x * x / ((2.0 * k + 1.0) * (2.0 * k + 2.0));
        ts *= -x * x / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
    return KTrigVal{c, s};
}
__host__ __device__ constexpr KTrigVal ktrig2pi(long long m, long long n)
{
    constexpr double pi4 = 0.78539816339744830962;  // pi / 4
    m %= n;
    if (m < 0) m += n;
    const long long o = (8 * m) / n;      // octant
    const long long r = 8 * m - o * n;    // angle = (pi/4) (o + r/n)
    double c = 0.0, s = 0.0;
    if ((o & 1) == 0) {
        const KTrigVal t = ksincos_octant(pi4 * (double)r / (double)n);
        switch (o / 2) {
        case 0: c = t.c; s = t.s; break;
        case 1: c = -t.s; s = t.c; break;
        case 2: c = -t.c; s = -t.s; break;
        default: c = t.s; s = -t.c; break;
        }
    } else {
        const KTrigVal t = ksincos_octant(pi4 * (double)(n - r) / (double)n);  // (o+1) pi/4 - angle
        switch ((o + 1) / 2) {
        case 1: c = t.s; s = t.c; break;
        case 2: c = -t.c; s = t.s; break;
        case 3: c = -t.s; s = -t.c; break;
        default: c = t.c; s = -t.s; break;
        }
    }
    return KTrigVal{c, s};
}
template <int N> struct KTrigTab {
    double c[N], s[N];
};
template <int N> __host__ __device__ constexpr KTrigTab<N> ktrig_tab()
{
    KTrigTab<N> t{};
    for (int m = 0; m < N; ++m) {
        const KTrigVal v = ktrig2pi(m, N);
        t.c[m] = v.c;
        t.s[m] = v.s;
    }
    return t;
}

// a * exp(-2 pi i m / R) for a compile-time m (after unrolling): exact for
// the multiples of a quarter turn
template <class C, class T, int R>
__device__ __forceinline__ C twiddle_const(C a, int m, const KTrigTab<R>& tw)
{
    if (m == 0) return a;
    if (4 * m == R) return mmi(a);                      // -i
    if (2 * m == R) return mk<C>(-a.x, -a.y);           // -1
    if (4 * m == 3 * R) return mk<C>(-a.y, a.x);        // +i
    return rot(a, (T)tw.c[m], (T)-tw.s[m]);
}

// Composite size R = R1 R2 on registers (Cooley-Tukey with n = R2 n1 + n2,
// k = k1 + R1 k2): R2 DFTs of size R1 over the inputs n2, n2 + R2, ...,
// the internal twiddles exp(-2 pi i n2 k1 / R), then R1 DFTs of size R2.
template <class C, class T, int R1, int R2> struct DftCT {
    static constexpr int R = R1 * R2;
    static __device__ __forceinline__ void run(C* v)
    {
        constexpr KTrigTab<R> tw = ktrig_tab<R>();
        C y[R];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            C a[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
            Dft<C, T, R1>::run(a);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = twiddle_const<C, T, R>(a[k1], (n2 * k1) % R, tw);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            C b[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) b[n2] = y[n2 * R1 + k1];
            Dft<C, T, R2>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
        }
    }
};
#define P3_DFT_CT(R, R1, R2)                                            \
    template <class C, class T> struct Dft<C, T, R> {                   \
        static __device__ __forceinline__ void run(C* v) { DftCT<C, T, R1, R2>::run(v); } \
    };
P3_DFT_CT(6, 2, 3)
P3_DFT_CT(9, 3, 3)
P3_DFT_CT(10, 2, 5)
P3_DFT_CT(12, 4, 3)
P3_DFT_CT(14, 2, 7)
P3_DFT_CT(15, 3, 5)
P3_DFT_CT(18, 2, 9)
P3_DFT_CT(20, 4, 5)
P3_DFT_CT(21, 3, 7)
P3_DFT_CT(24, 8, 3)
P3_DFT_CT(25, 5, 5)
P3_DFT_CT(27, 3, 9)
P3_DFT_CT(28, 4, 7)
#undef P3_DFT_CT

}  // namespace p3
