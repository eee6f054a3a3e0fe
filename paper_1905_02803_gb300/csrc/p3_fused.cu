// Plane-fused X + Y stages (Sect. 2 stages one and two, done z-plane by
// z-plane so the second reads the first one's output from L2).
//
// A z-plane of the complex array (H x Ny values, 4.2 MB at 1024^2 FP32) is
// written by the X stage and read back at once by the Y stage; with every
// plane's Y tiles queued right behind its X tiles, a plane is consumed while
// it is still in the 129 MB L2, so the pair of stages moves the real array
// once and the complex array once instead of the complex array three times.
// One persistent launch (a CTA per resident slot, cooperative so all are
// co-resident) takes tasks in ticket order from an atomic counter, the
// consumers of a plane `lag` planes behind its producers so that they
// rarely wait; a task only ever waits for tasks with smaller tickets, which
// running CTAs already hold, so the queue always drains.  Waits are bounded: after spin_limit
// polls a CTA records the failure in *err, skips the task and carries on.
#include "p3_pow2.cuh"

namespace p3 {

namespace {
using namespace pw;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// Tiles of the transposed-plane layout (planes stored [x][y], y fastest, so
// every Y line is contiguous).  The X tiles move their rows through shared
// memory once, to write (or read) them as B-wide runs across the tile's
// rows; the Y tiles are row-style: contiguous lines, exchanges private to a
// line's warp, no block barrier.
// ---------------------------------------------------------------------------
template <int B> __device__ __forceinline__ int tsw(int k) { return (k >> (B >= 16 ? 0 : B == 8 ? 1 : 2)) & (B - 1); }

// X r2c of rows y0 .. y0 + B - 1 of one plane (real rows L0 + l of the X
// stage's input), written to plane[k * ny + y0 + l].  The rows' last-pass
// outputs go to shared memory once; the store lanes (across rows) read
// Z[k] and Z[N-k] there and write the post-twiddled F[k] straight to the
// plane.  Row pitch RPX = 16/B (mod 16) complex keeps those cross-row reads
// on distinct banks (a half-warp covers the B rows at 16/B consecutive k).
template <int N, int E, int B> __host__ __device__ constexpr int xt_pitch()
{
    return (N + N / E) + ((16 / B - (N + N / E) % 16) % 16 + 16) % 16;
}

template <typename T, int N, int E, int B, int LP>
__device__ __forceinline__ void xr2c_tile_t(const StageArgs& a, long long L0, typename CxT<T>::t* plane, int y0,
                                            int ny, typename CxT<T>::t* s)
{
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS, NT = B * TPL, RPX = xt_pitch<N, E, B>();
    typedef RowSlot<N, E> S;
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long L = L0 + l;
    const C* tw2 = static_cast<const C*>(a.tw2);
    C* srow = s + l * RPX;
    C v[E];
    typedef PassIdx<N, E, 0> P0;
    typedef PassIdx<N, E, NP - 1> PLast;
    {
        const C* src = reinterpret_cast<const C*>(static_cast<const T*>(a.src) + L * a.in.lstride);
#pragma unroll
        for (int b = 0; b < P0::BM; ++b)
#pragma unroll
            for (int r = 0; r < P0::R; ++r) v[b * P0::R + r] = ldx<LP>(src + t + P0::in_K(b, r));
    }
    pass_compute<C, T, N, E, 0>(v, t, tw2, 2);
    RowRest<C, T, N, E, 1, NP, 0>::run(v, srow, t, static_cast<const C*>(a.twr));
    row_sync<TPL>();
    {
        const int u = PLast::out_u(t);
#pragma unroll
        for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
            for (int r = 0; r < PLast::R; ++r) srow[S::at_k(u, PLast::out_K(b, r), PLast::OUT_UA)] = v[b * PLast::R + r];
    }
    __syncthreads();  // the store lanes read every row of the tile
    // F[k] = (Z[k] + conj Z[N-k]) / 2 - i exp(-2 pi i k / 2N) (Z[k] - conj Z[N-k]) / 2
    static_assert(NT % B == 0, "store lanes keep their row");
    const int ll = tid % B;
    const C* zr = s + ll * RPX;
    C* dst = plane + y0 + ll;
    for (int k = tid / B; k <= N; k += NT / B) {
        const C zk = zr[S::at(k == N ? 0 : k)];
        const C zm = cnj(zr[S::at(k == 0 ? 0 : N - k)]);
        const C p = mul(ldg(tw2 + k), sub(zk, zm));
        dst[(long long)k * ny] = mk<C>((T)0.5 * (zk.x + zm.x + p.y), (T)0.5 * (zk.y + zm.y - p.x));
    }
}

// X c2r of rows y0 .. y0 + B - 1 of one plane, read from plane[k * ny + y0 + l]
// (real rows L0 + l of the X stage's output).
template <typename T, int N, int E, int B, int SP>
__device__ __forceinline__ void xc2r_tile_t(const StageArgs& a, long long L0, const typename CxT<T>::t* plane, int y0,
                                            int ny, typename CxT<T>::t* s)
{
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS, NT = B * TPL;
    constexpr int H = N + 1, LPT = (H * B + NT - 1) / NT;
    typedef RowSlot<N, E> S;
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const long long L = L0 + l;
    const C* tw2 = static_cast<const C*>(a.tw2);
    {
        static_assert(NT % B == 0, "load lanes keep their row");
        const int ll = tid % B;
        const C* src = plane + y0 + ll;
        C w[LPT];
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int k = tid / B + j * (NT / B);
            if (k <= N) w[j] = __ldcg(src + (long long)k * ny);
        }
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int k = tid / B + j * (NT / B);
            if (k <= N) s[k * B + (ll ^ tsw<B>(k))] = w[j];
        }
    }
    __syncthreads();
    C v[E];
    typedef PassIdx<N, E, 0> P0;
    typedef PassIdx<N, E, NP - 1> PLast;
    // Z[k] = (F[k] + conj F[N-k]) + i (F[k] - conj F[N-k]) exp(+2 pi i k / 2N),
    // imaginary parts of F[0] and F[N] dropped; inverse via swp
#pragma unroll
    for (int b = 0; b < P0::BM; ++b)
#pragma unroll
        for (int r = 0; r < P0::R; ++r) {
            const int k = t + P0::in_K(b, r);
            C A = s[k * B + (l ^ tsw<B>(k))];
            C Bc = cnj(s[(N - k) * B + (l ^ tsw<B>(N - k))]);
            if (k == 0) {
                A.y = (T)0;
                Bc.y = (T)0;
            }
            const C ze = add(A, Bc);
            const C zo = mul(sub(A, Bc), cnj(ldg(tw2 + k)));
            v[b * P0::R + r] = swp(mk<C>(ze.x - zo.y, ze.y + zo.x));
        }
    __syncthreads();  // the exchange rows overlap the transposed tile
    pass_compute<C, T, N, E, 0>(v, t, tw2, 2);
    RowRest<C, T, N, E, 1, NP, 0>::run(v, s + l * S::RP, t, static_cast<const C*>(a.twr));
    C* dst = reinterpret_cast<C*>(static_cast<T*>(a.dst) + L * a.out.lstride);
    const int u = PLast::out_u(t);
#pragma unroll
    for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
        for (int r = 0; r < PLast::R; ++r) stx<SP>(dst + u + PLast::out_K(b, r), swp(v[b * PLast::R + r]));
}

// Complex FFT of the contiguous lines line0 .. line0 + B - 1 (< nlines) of
// `base` (pitch N), in place.
template <typename T, int N, int E, int B, bool INV, int LP, int SP>
__device__ __forceinline__ void line_tile(const StageArgs& a, typename CxT<T>::t* base, int line0, int nlines,
                                          typename CxT<T>::t* s)
{
    typedef typename CxT<T>::t C;
    typedef P2<N, E> PL;
    constexpr int TPL = PL::TPL, NP = PL::NPASS;
    typedef RowSlot<N, E> S;
    const int tid = threadIdx.x, t = tid % TPL, l = tid / TPL;
    const int line = line0 + l;
    const bool valid = line < nlines;
    const C zero = mk<C>((T)0, (T)0);
    const C* tw = static_cast<const C*>(a.tw);
    C* p = base + (long long)(valid ? line : 0) * N;
    C v[E];
    typedef PassIdx<N, E, 0> P0;
    typedef PassIdx<N, E, NP - 1> PLast;
#pragma unroll
    for (int b = 0; b < P0::BM; ++b)
#pragma unroll
        for (int r = 0; r < P0::R; ++r) {
            const C x = valid ? ldx<LP>(p + t + P0::in_K(b, r)) : zero;
            v[b * P0::R + r] = INV ? swp(x) : x;
        }
    pass_compute<C, T, N, E, 0>(v, t, tw, 1);
    RowRest<C, T, N, E, 1, NP, 0>::run(v, s + l * S::RP, t, static_cast<const C*>(a.twr));
    if (valid) {
        const int u = PLast::out_u(t);
#pragma unroll
        for (int b = 0; b < PLast::BM; ++b)
#pragma unroll
            for (int r = 0; r < PLast::R; ++r) {
                const C x = v[b * PLast::R + r];
                stx<SP>(p + u + PLast::out_K(b, r), INV ? swp(x) : x);
            }
    }
}

// Row / column tile shapes of the fused kernel: NT threads for both.
template <typename T> __host__ __device__ constexpr int fx_E(int N) { return row_E<T>(N); }
template <typename T> __host__ __device__ constexpr int fx_B(int N, int NT) { return NT / (N / fx_E<T>(N)); }
template <typename T> __host__ __device__ constexpr int fy_E(int N) { return col_E<T>(N, 0); }
template <typename T> __host__ __device__ constexpr int fy_B(int N, int NT) { return NT / (N / fy_E<T>(N)); }

// line tiles (transposed planes): row-style, E as for rows
template <typename T> __host__ __device__ constexpr int fl_E(int N) { return row_E<T>(N); }
template <typename T> __host__ __device__ constexpr int fl_B(int N, int NT) { return NT / (N / fl_E<T>(N)); }

template <typename T, int NX, int NY, int NT, bool TP>
__host__ __device__ constexpr size_t fused_smem()
{
    typedef typename CxT<T>::t C;
    const size_t bx = (size_t)fx_B<T>(NX, NT);
    size_t row = bx * (size_t)(NX + NX / fx_E<T>(NX) + 1) * sizeof(C);
    if (TP && bx * (size_t)(NX + 1) * sizeof(C) > row) row = bx * (size_t)(NX + 1) * sizeof(C);
    if (TP && bx * (size_t)xt_pitch<NX, fx_E<T>(NX), fx_B<T>(NX, NT)>() * sizeof(C) > row)
        row = bx * (size_t)xt_pitch<NX, fx_E<T>(NX), fx_B<T>(NX, NT)>() * sizeof(C);
    const size_t col = TP ? (size_t)fl_B<T>(NY, NT) * (size_t)(NY + NY / fl_E<T>(NY) + 1) * sizeof(C)
                          : (size_t)fy_B<T>(NY, NT) * (size_t)col_smem_slots<T, NY>() * sizeof(C);
    return row > col ? row : col;
}

// Threads per CTA of the fused kernels: four 128-thread CTAs per SM with
// transposed planes (measured faster than two of 256), two of 256 otherwise.
#ifndef P3_FUSED_NT
#define P3_FUSED_NT 256
#endif
#ifndef P3_FUSED_NT_TP
#define P3_FUSED_NT_TP 128
#endif
// Resident CTAs per SM the transposed-plane kernels are compiled for: five
// forward (96 registers, measured 2.68 -> 2.61 ms at 1024^3), four inverse
// (its c2r tile spills at 96)
#ifndef P3_FUSED_MINB_TP_FWD
#define P3_FUSED_MINB_TP_FWD 5
#endif
#ifndef P3_FUSED_MINB_TP_INV
#define P3_FUSED_MINB_TP_INV 4
#endif

// NX: half length of the real X rows (complex points), NY: Y line length,
// NT: threads per CTA (both tile kinds), TP: transposed planes.
template <typename T, int NX, int NY, int DIR, int NT, bool TP>
__global__ void __launch_bounds__(NT, (TP ? (DIR == 0 ? P3_FUSED_MINB_TP_FWD : P3_FUSED_MINB_TP_INV) : 512 / NT))
    plane_kernel(const __grid_constant__ PlaneArgs f)
{
    typedef typename CxT<T>::t C;
    constexpr int EX = fx_E<T>(NX), BX = fx_B<T>(NX, NT);
    constexpr int EY = TP ? fl_E<T>(NY) : fy_E<T>(NY), BY = TP ? fl_B<T>(NY, NT) : fy_B<T>(NY, NT);
    static_assert(BX >= 1 && BY >= 1 && BX * (NX / EX) == NT && BY * (NY / EY) == NT, "fused tiles take NT threads");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    __shared__ unsigned s_task;
    __shared__ int s_ok;

    const unsigned first = DIR == 0 ? f.xt : f.yt;   // producers per plane
    const unsigned second = DIR == 0 ? f.yt : f.xt;  // consumers per plane
    const unsigned per = first + second;
    const unsigned np = (unsigned)f.nplanes, lag = (unsigned)f.lag;
    const unsigned total = np * per;
    const unsigned pro = lag * first, mid = (np - lag) * per;
    // thread 0 claims the next ticket while the current task runs (a CTA
    // holds at most one unstarted ticket, larger than its current one, so
    // the smallest unfinished ticket can always proceed)
    unsigned next = 0;
    if (threadIdx.x == 0) next = atomicAdd(f.ctr, 1u);
    for (;;) {
        if (threadIdx.x == 0) s_task = next;
        __syncthreads();
        const unsigned tk = s_task;
        if (tk >= total) return;
        if (threadIdx.x == 0) next = atomicAdd(f.ctr, 1u);
        // ticket order: producers of planes 0 .. lag-1; then for each plane
        // p = lag .. np-1 its producers followed by the consumers of plane
        // p - lag; then the consumers of the last lag planes
        unsigned plane, r;
        bool prod;
        if (tk < pro) {
            plane = tk / first;
            r = tk % first;
            prod = true;
        } else if (tk - pro < mid) {
            const unsigned u = tk - pro, sl = u / per, q = u % per;
            prod = q < first;
            plane = prod ? lag + sl : sl;
            r = prod ? q : q - first;
        } else {
            const unsigned v = tk - pro - mid;
            plane = np - lag + v / second;
            r = v % second;
            prod = false;
        }
        // Consumer tiles whose lines each belong to one warp (forward Y tiles
        // of transposed planes, lines of at most 32 lanes) wait warp by warp
        // and need no block barrier; other consumers wait as a block.
        constexpr bool WARP_Y = TP && DIR == 0 && (NY / EY) <= 32;
        if (!prod && WARP_Y) {
            int ok = 1;
            if ((threadIdx.x & 31) == 0) {
                const unsigned* done = f.ctr + 1 + plane;
                const unsigned need = first + f.extra;
                unsigned it = 0;
                while (ld_acquire(done) < need) {
                    if (++it > f.spin_limit || ld_acquire(f.err) != 0) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
                if (!ok) atomicOr(f.err, 1u);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) continue;  // the output is invalid; the host reads *err
        } else if (!prod) {
            if (threadIdx.x == 0) {
                const unsigned* done = f.ctr + 1 + plane;
                const unsigned need = first + f.extra;
                unsigned it = 0;
                int ok = 1;
                while (ld_acquire(done) < need) {
                    if (++it > f.spin_limit || ld_acquire(f.err) != 0) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
                if (!ok) atomicOr(f.err, 1u);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) continue;  // the output is invalid; the host reads *err
        }
        const bool isx = (DIR == 0) == prod;
        // Cache policies: the data that crosses HBM once (the real array, and
        // the complex plane once its second stage is done) streams with
        // evict-first hints; the plane between the two stages stays in L2,
        // and is read through L2 only (other CTAs wrote it).
        if constexpr (TP) {
            // planes [x][y]: X tiles of BX rows (ny a multiple of BX), Y
            // tiles of BY contiguous lines
            C* pl = static_cast<C*>(DIR == 0 ? f.x.dst : const_cast<void*>(f.x.src)) + (long long)plane * f.yoff;
            const long long L0 = (long long)plane * f.rows + (long long)r * BX;
            if (isx) {
                if constexpr (DIR == 0)
                    xr2c_tile_t<T, NX, EX, BX, LD_CS>(f.x, L0, pl, (int)r * BX, f.rows, s);
                else
                    xc2r_tile_t<T, NX, EX, BX, ST_CS>(f.x, L0, pl, (int)r * BX, f.rows, s);
            } else {
                if constexpr (DIR == 0)
                    line_tile<T, NY, EY, BY, false, LD_CG, ST_CS>(f.y, pl, (int)r * BY, NX + 1, s);
                else
                    line_tile<T, NY, EY, BY, true, LD_DEF, ST_DEF>(f.y, pl, (int)r * BY, NX + 1, s);
            }
        } else if (isx) {
            const long long L0 = (long long)plane * f.rows + (long long)r * BX;
            if constexpr (DIR == 0)
                row_tile<T, NX, EX, BX, 0, LD_CS, ST_DEF>(f.x, L0, (long long)(plane + 1) * f.rows, s);
            else
                row_tile<T, NX, EX, BX, 1, LD_CG, ST_CS>(f.x, L0, (long long)(plane + 1) * f.rows, s);
        } else {
            if constexpr (DIR == 0)
                col_tile<T, NY, EY, BY, 0, false, 0, LD_CG, ST_CS>(f.y, r, (long long)plane * f.yoff, s);
            else
                col_tile<T, NY, EY, BY, 0, true, 0, LD_DEF, ST_DEF>(f.y, r, (long long)plane * f.yoff, s);
        }
        // a producer counts its tile once every thread's stores are issued;
        // consumers go straight on (the barrier at the top of the loop keeps
        // the next tile from reusing shared memory too early)
        if (prod) {
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(f.ctr + 1 + plane, 1u);
            }
        }
    }
}

template <int NX, int NY> void* pick_dir(int dir, bool tp)
{
    if (tp)
        return dir == 0 ? (void*)plane_kernel<float, NX, NY, 0, P3_FUSED_NT_TP, true>
                        : (void*)plane_kernel<float, NX, NY, 1, P3_FUSED_NT_TP, true>;
    return dir == 0 ? (void*)plane_kernel<float, NX, NY, 0, P3_FUSED_NT, false>
                    : (void*)plane_kernel<float, NX, NY, 1, P3_FUSED_NT, false>;
}
template <int NX> void* pick_ny(int ny, int dir, bool tp)
{
    switch (ny) {
    case 256: return pick_dir<NX, 256>(dir, tp);
    case 512: return pick_dir<NX, 512>(dir, tp);
    case 1024: return pick_dir<NX, 1024>(dir, tp);
    case 2048: return pick_dir<NX, 2048>(dir, tp);
    default: return nullptr;
    }
}
// FP32 row half-lengths and column lengths with a fused kernel
void* pick(int nx, int ny, int dir, bool tp)
{
    switch (nx) {
    case 256: return pick_ny<256>(ny, dir, tp);
    case 512: return pick_ny<512>(ny, dir, tp);
    case 1024: return pick_ny<1024>(ny, dir, tp);
    default: return nullptr;
    }
}
template <int NT, bool TP> size_t smem_nt(int nx, int ny)
{
    size_t m = 0;
#define P3_SM(A, B) if (nx == A && ny == B) m = fused_smem<float, A, B, NT, TP>();
    P3_SM(256, 256) P3_SM(256, 512) P3_SM(256, 1024)
    P3_SM(512, 256) P3_SM(512, 512) P3_SM(512, 1024)
    P3_SM(1024, 256) P3_SM(1024, 512) P3_SM(1024, 1024)
    P3_SM(256, 2048) P3_SM(512, 2048) P3_SM(1024, 2048)
#undef P3_SM
    return m;
}

}  // namespace

bool fused_configure(PlaneArgs& f, const StageArgs& x, const StageArgs& y, int dir, size_t csize, bool tp)
{
    if (csize != 8 || x.blue || y.blue || y.tc) return false;
    const bool xok = dir == 0 ? x.op == OP_R2C_HALF : x.op == OP_C2R_HALF;
    if (!xok || y.op != OP_C2C || x.kern != (dir == 0 ? KIND_ROW_R2C : KIND_ROW_C2R) || y.kern != KIND_COL_DD)
        return false;
    void* fn = pick(x.nfft, y.nfft, dir, tp);
    if (!fn) return false;
    const int nt = tp ? P3_FUSED_NT_TP : P3_FUSED_NT;
    const size_t smem = tp ? smem_nt<P3_FUSED_NT_TP, true>(x.nfft, y.nfft) : smem_nt<P3_FUSED_NT, false>(x.nfft, y.nfft);
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (!coop || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    memset(&f, 0, sizeof(f));
    f.x = x;
    f.y = y;
    f.dir = dir;
    f.kx = x.nfft;
    f.ky = y.nfft;
    f.smem = smem;
    f.nt = nt;
    f.tp = tp ? 1 : 0;
    f.bx = fx_B<float>(x.nfft, nt);
    f.by = tp ? fl_B<float>(y.nfft, nt) : fy_B<float>(y.nfft, nt);
    if (y.nfft % f.bx) return false;  // X tiles of transposed planes are whole
    f.grid = per_sm * sms;
    f.spin_limit = 1u << 23;
    f.lag = 1;
    return true;
}

cudaError_t fused_prepare() { return cudaSuccess; }

cudaError_t fused_launch(const PlaneArgs& f, cudaStream_t s)
{
    void* fn = pick(f.kx, f.ky, f.dir, f.tp != 0);
    if (!fn || !f.ctr || !f.err) return cudaErrorInvalidValue;
    if (f.x.nlines <= 0 || f.nplanes <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(f.ctr, 0, sizeof(unsigned) * (size_t)(1 + f.nplanes), s);
    if (e != cudaSuccess) return e;
    PlaneArgs m = f;
    line_magic(m.x.in, m.x.nlines);
    line_magic(m.x.out, m.x.nlines);
    line_magic(m.y.in, m.y.nlines);
    line_magic(m.y.out, m.y.nlines);
    void* args[] = {&m};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)f.grid), dim3((unsigned)f.nt), args, f.smem, s);
}

}  // namespace p3
