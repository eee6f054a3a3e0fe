// Internal declarations shared by the plan code (p3_plan.cu) and the stage
// kernels (p3_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace p3 {

// Largest radix sequence a line plan can hold (mixed 2/3/5/7 factorizations
// of lengths <= 4096 have at most 12 prime factors).
constexpr int kMaxPasses = 14;
// Generic kernel: about this many points of a line per thread (threads per
// line = ceil(n / kVmax); the pass loops take any count).
#ifndef P3_GEN_VMAX
#define P3_GEN_VMAX 16
#endif
constexpr int kVmax = P3_GEN_VMAX;
// Largest composite radix (register butterflies 6 .. 28) of the FP32 generic
// kernel; the plan's factorisation uses the same bound.  16 (composites 6, 9,
// 10, 12, 14, 15) keeps the kernel free of spills at 85 registers and
// measured best on the 64-grid batch (6.89 ms, against 7.15 ms with all
// composites up to 28, whose larger butterflies spill).
#ifndef P3_GEN_MAXCR
#define P3_GEN_MAXCR 16
#endif
constexpr int kMaxCompositeRadix = P3_GEN_MAXCR;
// Threads per CTA never exceed this (matches __launch_bounds__).
constexpr int kMaxThreads = 256;
// Threads per CTA of the generic stage kernel (its own launch bounds).
#ifndef P3_GEN_MAXT
#define P3_GEN_MAXT 256
#endif
constexpr int kGenThreads = P3_GEN_MAXT;
// Longest native line; Bluestein lines need a padded length <= this too.
constexpr int kMaxLine = 4096;

// Line L, element e of a strided batch lives at
//   (L / per) * gstride + (L % per) * lstride + e * es
// counted in elements of the array's type (real or complex).
struct LineMap {
    long long per, gstride, lstride, es;
    // L / per as a multiply-high when pm != 0 (see line_magic)
    unsigned pm;
    int ps;
};

// Fills m.pm / m.ps so that L / per = (L * pm) >> ps for every line
// 0 <= L < nlines (Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994, Sect. 4, with 31-bit numerators:
// l = ceil(log2 per), pm = floor(2^(31+l) / per) + 1 < 2^32, ps = 31 + l);
// pm = 0 (plain division) when per or nlines does not fit in 31 bits.
inline void line_magic(LineMap& m, long long nlines)
{
    m.pm = 0;
    m.ps = 0;
    if (m.per < 1 || m.per >= (1LL << 31) || nlines > (1LL << 31)) return;
    int l = 0;
    while ((1LL << l) < m.per) ++l;
    m.pm = (unsigned)((1ULL << (31 + l)) / (unsigned long long)m.per + 1ULL);
    m.ps = 31 + l;
}

// Stage kernel families (StageArgs::kern).
enum KernelKind : int {
    KIND_GENERIC = 0,  // runtime mixed radix / Bluestein, any length
    KIND_COL_DD = 1,   // power of two, strided lines, HBM -> regs -> HBM
    KIND_COL_DS = 2,   // power of two, strided in, element-contiguous out (ZYX store)
    KIND_COL_SD = 3,   // power of two, element-contiguous in (ZYX load), strided out
    KIND_ROW_R2C = 4,  // power-of-two half length, X-stage real-to-complex
    KIND_ROW_C2R = 5,  // power-of-two half length, X-stage complex-to-real
};

enum StageOp : int {
    OP_C2C = 0,       // complex line -> complex line
    OP_R2C_HALF = 1,  // even Nx: length Nx/2 complex FFT of (f[2j], f[2j+1]) + real split
    OP_R2C_PAIR = 2,  // odd Nx: two real rows as one complex line f1 + i f2, FFT, both spectra split off
    OP_C2R_HALF = 3,  // even Nx: Hermitian pre-twiddle + length Nx/2 complex FFT
    OP_C2R_PAIR = 4,  // odd Nx: two half spectra as one line X1 + i X2 (both Hermitian-extended),
                      // FFT, real and imaginary parts
    OP_DCT1 = 5,      // Chebyshev: even extension to 2M points, FFT, first M+1 bins
    OP_COPY = 6,      // empty transform (re-orientation only)
    OP_DST1 = 7,      // sine: odd extension to 2(n+1) points, FFT, i times bins 1..n
};

// Everything one stage kernel launch needs (passed by value).
// Constants of one Stockham pass of the generic kernel (radix R after
// passes whose radices multiply to Ns), computed on the host at launch by
// generic_consts so that no thread divides by a run-time value.
struct PassConsts {
    int tstep;    // twiddle-table index of one unit of j mod Ns: (n / (Ns R)) * ts
    int dq, dr;   // tpl / Ns, tpl mod Ns (a thread's step through the butterflies)
    unsigned pm;  // t / Ns = (t * pm) >> ps (see line_magic)
    int ps;
};

struct StageArgs {
    // TMA descriptor of the input tile (tma = 1): lines as the inner
    // dimension, line elements as the outer one; encoded per call with the
    // call's source pointer
    CUtensorMap tmap;
    const void* src;
    void* dst;
    LineMap in, out;
    long long nlines;
    long long nrows;   // pair ops: real rows (line L holds rows 2L and 2L + 1 < nrows)
    int op;
    int n_in, n_out;   // points read / written per line
    int nfft;          // length of the complex DFT done on each line
    int sign;          // -1 forward, +1 inverse
    int B;             // lines per CTA (power of two)
    int LDB;           // shared-memory pitch between consecutive elements of a line
    int tpl;           // threads per line
    int in_elem_fast;  // 1: global input has es == 1 (lanes walk elements)
    int out_elem_fast; // 1: global output has es == 1
    // native Stockham passes over nfft points
    int npass;
    int rad[kMaxPasses];
    const void* tw;    // tw[k] = exp(-2 pi i k / twn), complex of the stage type
    int twn;
    const void* tw2;   // real-split twiddles exp(-2 pi i k / Nx) (R2C/C2R_HALF), length Nx
    const void* twr;   // power-of-two lines: per-pass twiddles laid out for row-style lanes
    // Bluestein (nfft not 7-smooth): DFT_nfft via padded length m
    int blue;
    int m;
    int mpass;
    int mrad[kMaxPasses];
    const void* chirp; // c[j] = exp(-pi i j^2 / nfft), j < nfft
    const void* bhat;  // DFT_m of the conjugate chirp filter, pre-scaled by 1/m
    const void* twm;   // exp(-2 pi i k / m), k < m
    PassConsts pc[kMaxPasses];   // per pass of rad (generic kernel; filled at launch)
    PassConsts mpc[kMaxPasses];  // per pass of mrad (Bluestein)
    size_t smem;       // dynamic shared memory bytes
    int threads;       // B * tpl
    int kern;          // KernelKind
    // 1: tensor-core split-precision kernel (p3_tc.cu)
    int tc;
    // 1: TMA-staged ZYX-store column kernel (input tile by tensor copies);
    // 2: row-style ZYX-load kernel with a bulk-copied input tile
    int tma;
    // status word of the plan: a bounded device wait that gave up ORs a bit in
    unsigned* err;
    // polls before a wait for a tensor / bulk copy gives up
    unsigned spin;
    // test mode (1): the copy barrier waits for one arrival more than the
    // copies make, so the wait runs out; the kernel then supplies the
    // missing arrival and waits for its copies before it leaves
    int wait_extra;
};

inline void pass_consts(PassConsts* pc, int n, int npass, const int* rad, int tpl, int ts)
{
    long long ns = 1;
    for (int p = 0; p < npass && p < kMaxPasses; ++p) {
        const long long R = rad[p] > 0 ? rad[p] : 1;
        pc[p].tstep = (int)((n / (ns * R)) * ts);
        pc[p].dq = (int)(tpl / ns);
        pc[p].dr = (int)(tpl % ns);
        LineMap m = LineMap{ns, 0, 0, 0};
        line_magic(m, 1LL << 31);
        pc[p].pm = m.pm;
        pc[p].ps = m.ps;
        ns *= R;
    }
}

// Fills the per-pass constants of a generic-kernel stage.
inline void generic_consts(StageArgs& a)
{
    pass_consts(a.pc, a.nfft, a.npass, a.rad, a.tpl, a.twn / (a.nfft > 0 ? a.nfft : 1));
    if (a.blue) pass_consts(a.mpc, a.m, a.mpass, a.mrad, a.tpl, 1);
}

// Launch one stage (defined in p3_kernels.cu).  Returns the launch error.
cudaError_t launch_stage_f32(const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_f64(const StageArgs& a, cudaStream_t s);
// One-time kernel attribute set-up for the current device (max dynamic smem).
cudaError_t prepare_kernels();

// Power-of-two specialised kernels (p3_pow2.cu): configure a stage for them
// (returns false when none applies), set them up, launch one stage.
bool pow2_configure(StageArgs& a, size_t csize, bool allow_tma);
// Encodes a.tmap for a stage with a.tma set, from a.src (p3_pow2.cu).
cudaError_t pow2_encode_tma(StageArgs& a);
cudaError_t pow2_prepare();
cudaError_t pow2_launch(const StageArgs& a, bool f32, cudaStream_t s);

// Fused X + Y stages over z-planes (p3_fused.cu).  One persistent launch
// whose CTAs take tasks from a queue in ticket order: the producer tasks of
// planes 0 .. lag-1, then for p = lag .. Nz-1 the producer tasks of plane p
// followed by the consumer tasks of plane p - lag, then the consumer tasks
// of the last lag planes.
// Forward the producers are X r2c row tiles and the consumers Y column tiles
// (in place); inverse the producers are Y column tiles and the consumers X
// c2r row tiles.  A consumer waits (bounded) until every producer of its
// plane has finished; the plane is then still in L2.
struct PlaneArgs {
    StageArgs x;          // the whole X stage (rows map over Ny*Nz rows)
    StageArgs y;          // the Y stage of one plane (H lines), in place
    int dir;              // 0 forward, 1 inverse
    int nplanes;          // Nz
    int xt, yt;           // X row tiles / Y column tiles per plane
    int rows;             // Ny: X rows per plane
    long long yoff;       // Ny * H: complex elements per plane
    unsigned* ctr;        // [0] ticket, [1 + p] producers done of plane p (zeroed before launch)
    unsigned* err;        // set non-zero when a wait gives up
    unsigned spin_limit;  // polls before a wait gives up
    unsigned extra;       // added to the producer count a consumer waits for (0; > 0 only in tests)
    int lag;              // consumers of plane p follow the producers of plane p + lag (1 <= lag <= nplanes)
    int grid;             // persistent CTAs
    int nt;               // threads per CTA
    int tp;               // 1: planes stored transposed, [x][y] (y fastest)
    int bx, by;           // rows per X tile, lines per Y tile
    size_t smem;
    int kx, ky;           // row / column line lengths (complex points)
};

// Returns true when a plane-fused kernel exists for these X and Y stages;
// fills f (except buffers and counters).
bool fused_configure(PlaneArgs& f, const StageArgs& x, const StageArgs& y, int dir, size_t csize, bool tp);
cudaError_t fused_prepare();
cudaError_t fused_launch(const PlaneArgs& f, cudaStream_t s);


// A stage of a plan configured for the generic kernel, with its buffer
// roles (0 input, 1 output, 2 workspace): the building block of the batched
// persistent launch.
struct GenericStage {
    StageArgs a;
    int src, dst;
};

// Batched persistent launch (p3_batch.cu builds the task table, the kernel
// is in p3_kernels.cu).  Every (plan, stage) of a direction is a task of
// ntiles tiles; task i owns tickets first .. first + ntiles - 1; tasks are
// ordered level by level (every plan's first stage, then every plan's
// second, ...), so a tile only waits for tiles of a lower level, which
// running CTAs already hold.
struct BatchTask {
    StageArgs a;        // generic-kernel stage; src and dst come from the call
    long long first;    // first ticket
    long long ntiles;
    int plan;           // row of the call's buffer table
    int src, dst;       // buffer roles
    int dep;            // task that must be finished first, or -1
};
constexpr int kBatchMaxPlans = 256;
// The scheduling fields of a task, in a compact array the CTAs search.
struct BatchMeta {
    unsigned first;   // first ticket
    unsigned ntiles;
    int dep;          // task that must be finished first, or -1
    int plan;         // row of the call's buffer table
    int src, dst;     // buffer roles
};
struct BatchLaunch {
    const BatchTask* tasks;  // device array, ntasks entries
    const BatchMeta* meta;   // device array, ntasks entries
    int ntasks;
    unsigned total;          // tickets
    unsigned* ctr;           // [0] next ticket, [1 + i] finished tiles of task i (zeroed before the launch)
    unsigned* err;           // set non-zero when a wait gives up
    unsigned spin_limit;     // polls before a wait gives up
    unsigned extra;          // added to the count a wait needs (0; > 0 only in tests)
    void* buf[kBatchMaxPlans][3];
};
// Resident CTAs of the batched kernel for `smem` bytes of dynamic shared
// memory (sets the kernel's shared-memory limit); 0 on failure.
int batch_grid(size_t smem);
cudaError_t batch_launch(const BatchLaunch& b, int grid, size_t smem, cudaStream_t s);

// Tensor-core split-precision kernels (p3_tc.cu): FP32 1024-point columns.
bool tc_configure(StageArgs& a, size_t csize);
cudaError_t tc_prepare();
cudaError_t tc_launch(const StageArgs& a, cudaStream_t s);

}  // namespace p3
