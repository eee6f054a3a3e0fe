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

// Row / column tile shapes of the fused kernel: NT threads for both.
template <typename T> __host__ __device__ constexpr int fx_E(int N) { return row_E<T>(N); }
template <typename T> __host__ __device__ constexpr int fx_B(int N, int NT) { return NT / (N / fx_E<T>(N)); }
template <typename T> __host__ __device__ constexpr int fy_E(int N) { return col_E<T>(N, 0); }
template <typename T> __host__ __device__ constexpr int fy_B(int N, int NT) { return NT / (N / fy_E<T>(N)); }

template <typename T, int NX, int NY, int NT>
__host__ __device__ constexpr size_t fused_smem()
{
    typedef typename CxT<T>::t C;
    const size_t row = (size_t)fx_B<T>(NX, NT) * (size_t)(NX + NX / fx_E<T>(NX) + 1) * sizeof(C);
    const size_t col = (size_t)fy_B<T>(NY, NT) * (size_t)col_smem_slots<T, NY>() * sizeof(C);
    return row > col ? row : col;
}

// Threads per CTA of each direction's fused kernel.
#ifndef P3_FUSED_NT_FWD
#define P3_FUSED_NT_FWD 256
#endif
#ifndef P3_FUSED_NT_INV
#define P3_FUSED_NT_INV 256
#endif

// NX: half length of the real X rows (complex points), NY: Y line length,
// NT: threads per CTA (both tile kinds).
template <typename T, int NX, int NY, int DIR, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) plane_kernel(const __grid_constant__ PlaneArgs f)
{
    typedef typename CxT<T>::t C;
    constexpr int EX = fx_E<T>(NX), BX = fx_B<T>(NX, NT);
    constexpr int EY = fy_E<T>(NY), BY = fy_B<T>(NY, NT);
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
        if (!prod) {
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
        if (isx) {
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
        __syncthreads();
        if (prod && threadIdx.x == 0) {
            __threadfence();
            atomicAdd(f.ctr + 1 + plane, 1u);
        }
    }
}

template <int NX, int NY> void* pick_dir(int dir)
{
    return dir == 0 ? (void*)plane_kernel<float, NX, NY, 0, P3_FUSED_NT_FWD>
                    : (void*)plane_kernel<float, NX, NY, 1, P3_FUSED_NT_INV>;
}
template <int NX> void* pick_ny(int ny, int dir)
{
    switch (ny) {
    case 256: return pick_dir<NX, 256>(dir);
    case 512: return pick_dir<NX, 512>(dir);
    case 1024: return pick_dir<NX, 1024>(dir);
    default: return nullptr;
    }
}
// FP32 row half-lengths and column lengths with a fused kernel
void* pick(int nx, int ny, int dir)
{
    switch (nx) {
    case 256: return pick_ny<256>(ny, dir);
    case 512: return pick_ny<512>(ny, dir);
    case 1024: return pick_ny<1024>(ny, dir);
    default: return nullptr;
    }
}
template <int NT> size_t smem_nt(int nx, int ny)
{
    size_t m = 0;
#define P3_SM(A, B) if (nx == A && ny == B) m = fused_smem<float, A, B, NT>();
    P3_SM(256, 256) P3_SM(256, 512) P3_SM(256, 1024)
    P3_SM(512, 256) P3_SM(512, 512) P3_SM(512, 1024)
    P3_SM(1024, 256) P3_SM(1024, 512) P3_SM(1024, 1024)
#undef P3_SM
    return m;
}

}  // namespace

bool fused_configure(PlaneArgs& f, const StageArgs& x, const StageArgs& y, int dir, size_t csize)
{
    if (csize != 8 || x.blue || y.blue || y.tc) return false;
    const bool xok = dir == 0 ? x.op == OP_R2C_HALF : x.op == OP_C2R_HALF;
    if (!xok || y.op != OP_C2C || x.kern != (dir == 0 ? KIND_ROW_R2C : KIND_ROW_C2R) || y.kern != KIND_COL_DD)
        return false;
    void* fn = pick(x.nfft, y.nfft, dir);
    if (!fn) return false;
    const int nt = dir == 0 ? P3_FUSED_NT_FWD : P3_FUSED_NT_INV;
    const size_t smem = dir == 0 ? smem_nt<P3_FUSED_NT_FWD>(x.nfft, y.nfft) : smem_nt<P3_FUSED_NT_INV>(x.nfft, y.nfft);
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
    f.bx = fx_B<float>(x.nfft, nt);
    f.by = fy_B<float>(y.nfft, nt);
    f.grid = per_sm * sms;
    f.spin_limit = 1u << 23;
    f.lag = 1;
    return true;
}

cudaError_t fused_prepare() { return cudaSuccess; }

cudaError_t fused_launch(const PlaneArgs& f, cudaStream_t s)
{
    void* fn = pick(f.kx, f.ky, f.dir);
    if (!fn || !f.ctr || !f.err) return cudaErrorInvalidValue;
    if (f.x.nlines <= 0 || f.nplanes <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(f.ctr, 0, sizeof(unsigned) * (size_t)(1 + f.nplanes), s);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<PlaneArgs*>(&f)};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)f.grid), dim3((unsigned)f.nt), args, f.smem, s);
}

}  // namespace p3
