/*
 * p3dfft_gb300.h -- C ABI of a single-GPU (GB300, sm_103a) library for the
 * 3D real-to-complex forward transform and its complex-to-real inverse, done
 * the way the P3DFFT paper (Pekurovsky, "P3DFFT: a framework for parallel
 * computations of Fourier transforms in three dimensions") describes: three
 * stages of batched 1D transforms -- X (real-to-complex), Y (complex) and Z
 * (complex FFT, Chebyshev or empty) -- with the paper's all-to-all
 * re-orientations between pencils turned into on-device transposes fused into
 * the stage kernels' loads and stores (Sect. 2, Fig. 2; Sect. 3.3).
 *
 * Conventions used by every call below.
 *
 * Arrays are C row-major with the rightmost index fastest; "dims" lists the
 * extents fastest first, as the paper's Table 1 lists L1, L2, L3.
 *   real input / output  (X-pencil, Table 1):   f[Nz][Ny][Nx]         dims {Nx, Ny, Nz}
 *   complex half-spectrum, H = floor(Nx/2) + 1 bins per X line (Sect. 3.2):
 *     P3_LAYOUT_XYZ  (STRIDE1 undefined):      F[Nz][Ny][H]          dims {H, Ny, Nz}
 *     P3_LAYOUT_ZYX  (STRIDE1 defined):        F[H][Ny][Nz]          dims {Nz, Ny, H}
 * Complex values are interleaved (re, im) pairs of the plan's precision.
 *
 * Transforms (Sect. 2, Sect. 3.1), both directions unnormalised:
 *   forward  F[kz][ky][kx] = sum_{x,y,z} f * exp(-2 pi i (kx x/Nx + ky y/Ny + kz z/Nz)),
 *            kx < H; a CHEB third dimension replaces the Z sum with the DCT-I
 *            Y_n = x_0 + (-1)^n x_M + 2 sum_{j=1}^{M-1} x_j cos(pi j n / M), M = Nz-1
 *            (real and imaginary parts alike; Gauss-Lobatto points
 *            z_j = cos(pi j / M)), a SINE third dimension the DST-I (the
 *            inverse applies the same DST-I again: scale 2(Nz+1)); an EMPTY
 *            dimension is the identity.
 *   inverse  the adjoint stages in reverse order with the + sign, the X stage
 *            being f[x] = Re sum_{k<H} w_k F[k] exp(+2 pi i k x / Nx) with
 *            w_0 = 1, w_{Nx/2} = 1 for even Nx, w_k = 2 otherwise (so the
 *            imaginary parts of each line's DC and Nyquist bins are ignored).
 *   A forward-inverse round trip returns the input times p3_plan_scale().
 *
 * Memory: every data pointer (inputs, outputs, workspace) is a caller-owned
 * device pointer of the device that was current at p3_plan_create, 16-byte
 * aligned.  The library allocates nothing per call; the plan owns only its
 * small twiddle / chirp tables (one cudaMalloc at creation).
 *
 * Execution: ftran / btran enqueue kernels on `stream` (a cudaStream_t; NULL
 * is the legacy default stream) and return without synchronising.  Inputs are
 * never written (except in place, see P3_FLAG_PADDED_REAL).  An output that
 * partly overlaps the input, or any buffer overlapping the workspace, is
 * rejected.  A plan is immutable after creation (except for the
 * optional timing events) and may be used from several threads with distinct
 * workspaces.  No call throws, aborts or prints.
 */
#ifndef P3DFFT_GB300_H
#define P3DFFT_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define P3_VERSION 1

typedef struct p3_plan_s* p3_plan;

typedef enum {
    P3_OK = 0,
    P3_ERR_INVALID = 1,     /* bad argument: NULL, misaligned, bad dims, overlap */
    P3_ERR_UNSUPPORTED = 2, /* valid request outside what this library implements */
    P3_ERR_NOMEM = 3,       /* host or device allocation at plan creation failed */
    P3_ERR_CUDA = 4,        /* a CUDA call or kernel launch failed */
    P3_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    P3_ERR_WORKSPACE = 6,   /* workspace required but NULL */
    P3_ERR_HOOK = 7         /* the user Z hook returned non-zero */
} p3_status;

/* Sect. 3.1: single and double precision. */
typedef enum { P3_F32 = 0, P3_F64 = 1 } p3_precision;

/* Sect. 3.1 / Sect. 5: Fourier, Chebyshev (DCT-I, third dimension only),
 * empty, and sine (DST-I of the Nz interior points of a Dirichlet grid,
 * Y_k = 2 sum_j x_j sin(pi (j+1)(k+1)/(Nz+1)), third dimension only; the
 * "sine" of Sect. 3.1's sine/cosine transforms). */
typedef enum { P3_FFT = 0, P3_CHEB = 1, P3_EMPTY = 2, P3_SINE = 3 } p3_ttype;

/* Plan flags (p3_plan_create). */
#define P3_FLAG_TC_SPLIT 1u
#define P3_FLAG_PADDED_REAL 2u
#define P3_FLAG_NO_FUSE 4u
#define P3_FLAG_TUNE 8u
#define P3_FLAG_NO_TMA 16u

/* Table 1: storage order of the Z-pencil complex array. */
typedef enum { P3_LAYOUT_ZYX = 0, P3_LAYOUT_XYZ = 1 } p3_layout;

/*
 * p3_plan_create -- build a plan for an Nx x Ny x Nz grid (Sect. 3.2: the
 * user sets the grid size; the library keeps its internal variables hidden).
 *   out        receives the plan handle (set to NULL on failure).
 *   nx,ny,nz   grid extents, each >= 1; Nz >= 2 when ttype[2] == P3_CHEB.
 *   prec       P3_F32 or P3_F64: the type of the data and of the arithmetic.
 *   ttype      per-dimension transform; ttype[0] must be P3_FFT (the X
 *              real-to-complex stage defines the path), ttype[1] P3_FFT or
 *              P3_EMPTY, ttype[2] P3_FFT, P3_CHEB, P3_SINE or P3_EMPTY.
 *   out_layout storage order of the complex array (Table 1).
 *   flags      0 or an OR of
 *              P3_FLAG_TC_SPLIT: run the FP32 1024-point Y / Z stages on the
 *                tensor cores in split precision (each FP32 operand split
 *                into a TF32 head and tail, three products accumulated in
 *                FP32).  No effect on other stages or precisions.
 *              P3_FLAG_PADDED_REAL (P3_LAYOUT_XYZ only, else
 *                P3_ERR_UNSUPPORTED): real arrays have rows of 2H values
 *                (f[Nz][Ny][2H], the last 2H - Nx of each row unused), the
 *                size of the complex array, so ftran and btran may run in
 *                place (in == out; Sect. 3.1 in-place transforms).  Neither
 *                direction then needs a workspace; out of place the inverse
 *                works in its output buffer and leaves the input untouched.
 *              P3_FLAG_NO_FUSE: launch the X and Y stages separately.  By
 *                default, where a fused kernel exists (FP32, even Nx with
 *                Nx/2 in {256, 512, 1024} and Ny in {256, 512, 1024, 2048},
 *                FFT in Y, no padded rows,
 *                no tensor-core split), the X and Y stages of each direction
 *                run as one persistent launch that works z-plane by z-plane
 *                so the second stage reads the first one's output from L2.
 *                Its CTAs wait on one another with bounded waits; see
 *                p3_plan_wait_status().
 *              P3_FLAG_TUNE: time candidates here and keep the fastest,
 *                the timings appearing in p3_plan_describe():
 *                - each stage of the generic kernel (lengths that are not
 *                  powers of two, Bluestein lines excepted) under a few
 *                  orders of its radices and tile heights (the same
 *                  transform, rounded in another order);
 *                - for each direction with a plane-fused launch, the fused
 *                  launch at a few queue lags and the separate X and Y
 *                  launches (the same result).
 *                Allocates buffers of the transform's size for the duration
 *                of the call, so plan creation takes milliseconds to a
 *                second.
 *              P3_FLAG_NO_TMA: load the Z stages' input tiles with ordinary
 *                loads instead of tensor-memory-access (TMA) copies: the
 *                forward ZYX-store stage (FP32 lines of 256 .. 2048 points)
 *                and the inverse ZYX-load stage when its lines lie one after
 *                another in memory (FP32 FFT lines of 256 .. 1024 points).
 * Any line length is accepted: lengths whose prime factors are 2, 3, 5, 7 run
 * natively; other lengths use Bluestein's chirp-z algorithm.  Lines longer
 * than 4096 points (2048 when Bluestein is needed) return P3_ERR_UNSUPPORTED.
 * Errors: P3_ERR_INVALID (NULL out/ttype, bad dims or enum, unknown flags),
 * P3_ERR_UNSUPPORTED, P3_ERR_NOMEM, P3_ERR_CUDA (no usable device).
 * Argument checks happen before any CUDA call.
 */
p3_status p3_plan_create(p3_plan* out, int nx, int ny, int nz, p3_precision prec,
                         const p3_ttype ttype[3], p3_layout out_layout, unsigned flags);

/* Releases the plan and its device tables.  NULL is accepted.  The caller
   must ensure no enqueued work still uses the plan. */
p3_status p3_plan_destroy(p3_plan plan);

/*
 * p3_ftran_r2c -- forward transform (R2C: X-pencil input, Z-pencil output,
 * Sect. 3.2).  in_real: Nx*Ny*Nz reals; out_cplx: H*Ny*Nz complex in the
 * plan's layout; workspace: p3_plan_workspace_bytes() bytes (may be NULL
 * when that is 0).  Errors: P3_ERR_INVALID (NULL plan/in/out, misaligned or
 * partly overlapping buffers), P3_ERR_UNSUPPORTED (in == out without
 * P3_FLAG_PADDED_REAL), P3_ERR_WORKSPACE,
 * P3_ERR_CUDA (launch failure; the stream state is then undefined).
 */
p3_status p3_ftran_r2c(p3_plan plan, const void* in_real, void* out_cplx,
                       void* workspace, void* stream);

/*
 * p3_btran_c2r -- inverse transform (C2R: Z-pencil input in the plan's
 * layout, X-pencil real output, Sect. 3.2).  in_cplx is not modified, which
 * is why the inverse needs a workspace.  Same errors as p3_ftran_r2c.
 */
p3_status p3_btran_c2r(p3_plan plan, const void* in_cplx, void* out_real,
                       void* workspace, void* stream);

/* Extents of the real (X-pencil) and complex (Z-pencil) arrays, fastest
   first, as in the header comment (Sect. 3.2 get-dimension routines). */
p3_status p3_plan_get_dims(p3_plan plan, int in_dims[3], int out_dims[3]);

/* Bytes of device workspace that ftran and btran need (the larger of the
   two); 0 when neither needs any. */
p3_status p3_plan_workspace_bytes(p3_plan plan, size_t* bytes);

/* Round-trip factor: btran(ftran(f)) = scale * f, the product over the
   dimensions of n (FFT), 2(n-1) (CHEB), 2(n+1) (SINE) or 1 (EMPTY)
   (Sect. 4.1); a Z hook's own factor is not included. */
p3_status p3_plan_scale(p3_plan plan, double* scale);

/*
 * Optional per-stage timing.  events: 8 cudaEvent_t handles (or NULL to turn
 * timing off).  ftran records events[0] before its first stage kernel and
 * events[i] after its i-th stage (i = 1..3); btran uses events[4..7] the same
 * way.  A direction with fewer than three stages records the remaining events
 * right after its last stage.  While events are set the plan must not be used
 * from two threads at once.
 */
p3_status p3_plan_set_stage_events(p3_plan plan, void* const* events, int n_events);

/*
 * Writes a one-line-per-stage description of the plan (kernel, line length,
 * radix sequence, lines per CTA, threads, shared memory, algorithmic bytes)
 * into buf (always NUL-terminated when len > 0).  P3_ERR_INVALID on NULL.
 */
p3_status p3_plan_describe(p3_plan plan, char* buf, size_t len);

/* Number of kernel launches one ftran (dir = 0) or btran (dir = 1) makes
   (with the Z hook set, if one is). */
p3_status p3_plan_launches(p3_plan plan, int dir, int* launches);

/*
 * The radix sequence a plan of precision prec gives the generic-kernel
 * stages of a line of n points (the Cooley-Tukey factorisation behind each
 * 1D FFT of Sect. 2; no device work, no GPU needed).  FP32 lengths with a
 * factor 3, 5 or 7 take the fewest passes over the native radices 2, 3, 4,
 * 5, 7, 8, 16 and the composite register butterflies up to 15; other
 * lengths take 16s first, then 8 / 4 / 2, then 3, 5, 7.  radices receives
 * up to cap entries (the largest radix first), *npass their count.
 * P3_ERR_UNSUPPORTED when n has a prime factor above 7 (such lines run
 * Bluestein's algorithm over a power-of-two length) or the sequence is
 * longer than cap; P3_ERR_INVALID for n < 2, a bad precision or NULL
 * pointers.
 */
p3_status p3_plan_factor(int n, p3_precision prec, int* radices, int cap, int* npass);

/*
 * Plane-fused X + Y launches (no paper counterpart; see P3_FLAG_NO_FUSE):
 * their CTAs wait, with a bounded number of polls, for the tiles of the same
 * z-plane that other CTAs compute.  A wait that gives up marks the plan's
 * device status word, skips its tile (that call's output is then invalid)
 * and lets the launch finish.  p3_plan_wait_status() synchronises with the
 * device, returns P3_ERR_TIMEOUT if any wait of this plan gave up since the
 * last check (and clears the mark), else P3_OK; P3_ERR_INVALID for NULL.
 * The waits of the Z kernels whose input tile arrives by tensor (TMA) or
 * bulk copies report the same way: a wait that gives up skips that tile
 * (the output is then invalid) after waiting, again bounded, for the copies
 * still in flight into the tile.
 */
p3_status p3_plan_wait_status(p3_plan plan);

/*
 * As p3_plan_wait_status(), but reports which kinds of wait gave up since
 * the last check: *flags = 0 when none did, else an OR of
 * P3_WAIT_FUSED_QUEUE (a plane-fused launch's wait for another tile) and
 * P3_WAIT_COPY (a Z kernel's wait for its tensor / bulk copies); the marks
 * are cleared.  Synchronises with the device.  P3_ERR_INVALID for NULL
 * arguments, P3_ERR_CUDA if the status word cannot be read.
 */
#define P3_WAIT_FUSED_QUEUE 1u
#define P3_WAIT_COPY 2u
p3_status p3_plan_wait_flags(p3_plan plan, unsigned* flags);

/*
 * Tuning of the plane-fused launches: the consumer tiles of z-plane p are
 * queued behind the producer tiles of plane p + lag.  A larger lag makes
 * waits rarer, a smaller one keeps fewer planes in flight in L2.  lag = 0
 * restores the plan's default; values above Nz act as Nz.  No effect on
 * plans without fused launches.  P3_ERR_INVALID for NULL or lag < 0.
 */
p3_status p3_plan_set_fused_lag(p3_plan plan, int lag);

/*
 * Test support for the bounded waits: spin_limit polls (>= 1; default
 * 2^23, over a second) before a plane-fused wait gives up (the Z kernels'
 * copy waits poll spin_limit / 2 times, each poll of the copy barrier may
 * itself pause briefly), and `extra`, which makes every wait run out
 * (0 by default): a fused wait then needs `extra` more finished tiles than
 * exist, and a copy wait one barrier arrival more than the copies make --
 * after giving up, the kernel makes that arrival itself and waits for its
 * copies, so the copies into shared memory have landed before it leaves.
 * This is how the tests check the error path.  P3_ERR_INVALID for NULL or
 * spin_limit == 0.
 */
p3_status p3_plan_set_wait_limits(p3_plan plan, unsigned spin_limit, unsigned extra);

/*
 * p3_z_hook -- a user transform in place of an EMPTY third dimension
 * (Sect. 3.1 and Sect. 5: the empty transform leaves the third dimension to a
 * transform of the user's own choice).  Called on the host, from inside
 * ftran / btran, with:
 *   data         device array of complex values (the plan's precision);
 *   n            Nz, points per Z line;
 *   nlines       H * Ny Z lines;
 *   line_stride, elem_stride   element j of line L is
 *                data[L * line_stride + j * elem_stride] (in complex
 *                elements): ZYX forward output (Nz, 1), otherwise XYZ order
 *                (1, H * Ny);
 *   dir          0 forward, 1 inverse;
 *   stream       the stream the caller passed to ftran / btran: the hook
 *                must enqueue its work on it (or synchronise with it) and
 *                may not block on later work of this call.
 * It transforms the lines in place and returns 0, or non-zero to stop the
 * call, which then returns P3_ERR_HOOK (stages already enqueued still run).
 * Forward, it runs on the output after the last stage; inverse, on a copy of
 * the input in the work buffer (workspace, or the output with
 * P3_FLAG_PADDED_REAL), before the inverse Y and X stages; the input is not
 * modified.
 */
typedef int (*p3_z_hook)(void* data, int n, long long nlines, long long line_stride, long long elem_stride,
                         int dir, void* stream, void* user);

/*
 * Sets (fn != NULL) or clears (fn == NULL) the plan's Z hook; user is passed
 * back to fn unchanged.  P3_ERR_INVALID for a NULL plan or a plan whose
 * ttype[2] is not P3_EMPTY.  The workspace size already covers the hook
 * mode.  Not thread-safe against concurrent ftran / btran on the same plan.
 */
p3_status p3_plan_set_z_hook(p3_plan plan, p3_z_hook fn, void* user);

/*
 * Batched execution of independent plans (no paper counterpart: many 3D
 * transforms per call), in one of two modes.
 *   Persistent (nstreams == 0): one kernel launch per call runs every stage
 *     of every plan.  Each stage is a task of the generic stage kernel; the
 *     launch's CTAs take (task, tile) tickets level by level (every plan's
 *     first stage, then every plan's second, ...), and a tile of a later
 *     stage waits, bounded, until the plan's previous stage has finished
 *     (see p3_batch_wait_status).  FP32 plans without a Z hook, at most 256
 *     plans.  The call's buffers are launch parameters, so consecutive calls
 *     never share host state, and the call can be captured into a CUDA
 *     graph.  Results equal each plan's own within rounding (the power-of-two
 *     and plane-fused kernels a plan may use alone are not used here).
 *   Streams (nstreams >= 1): the plans' own launches spread over nstreams
 *     internal streams (largest plans first, each to the least loaded
 *     stream), so the launches of different plans overlap on the GPU;
 *     results equal each plan's own bit for bit.
 *
 * p3_batch_create: plans (nplans >= 1, all created on the current device;
 *   the batch keeps the handles, not copies: destroy the batch first),
 *   nstreams >= 0 (capped at nplans).  Creates the streams and events, or
 *   the persistent mode's task tables (device memory owned by the batch).
 *   P3_ERR_INVALID on bad arguments, P3_ERR_UNSUPPORTED when the persistent
 *   mode cannot take a plan (FP64, a Z hook, more than 256 plans),
 *   P3_ERR_NOMEM / P3_ERR_CUDA if the batch's resources cannot be created.
 * p3_batch_ftran_r2c / p3_batch_btran_c2r: arrays of nplans pointers in
 *   plan order: in[i], out[i], ws[i] as p3_ftran_r2c / p3_btran_c2r take
 *   them for plan i (ws may be NULL when no plan needs a workspace, and
 *   ws[i] NULL for plans that need none).  Every buffer must be distinct
 *   from every other plan's (the plans run concurrently).  Stream-ordered on
 *   `stream`: the batch starts after the work already on `stream` and
 *   `stream` continues only after every plan finished; capturable into a
 *   CUDA graph.  Returns the first error of a plan; plans before it were
 *   enqueued and are still joined back into `stream`.
 */
typedef struct p3_batch_s* p3_batch;
p3_status p3_batch_create(p3_batch* out, int nplans, const p3_plan* plans, int nstreams);
p3_status p3_batch_destroy(p3_batch batch);
p3_status p3_batch_ftran_r2c(p3_batch batch, const void* const* in, void* const* out, void* const* ws,
                             void* stream);
p3_status p3_batch_btran_c2r(p3_batch batch, const void* const* in, void* const* out, void* const* ws,
                             void* stream);

/* Persistent mode: P3_ERR_TIMEOUT if a tile's bounded wait for the previous
   stage of its plan gave up since the last check (that call's outputs are
   invalid; the mark is cleared), else P3_OK.  Synchronises with the device.
   Stream mode: P3_OK (each plan reports through p3_plan_wait_status).
   P3_ERR_INVALID for NULL. */
p3_status p3_batch_wait_status(p3_batch batch);

/* Persistent mode, as p3_plan_set_wait_limits: spin_limit polls before a
   tile's wait gives up (default 2^23, over a second), and `extra` finished
   tiles more than exist needed by every wait (0 by default; > 0 makes every
   wait run out, for tests of the error path).  P3_ERR_INVALID for NULL or
   spin_limit == 0. */
p3_status p3_batch_set_wait_limits(p3_batch batch, unsigned spin_limit, unsigned extra);

/* Kernel launches one batch call makes in direction dir (0 forward, 1
   inverse): 1 in persistent mode, the plans' launches summed in stream
   mode (counter memsets are not launches).  P3_ERR_INVALID on bad
   arguments. */
p3_status p3_batch_launches(p3_batch batch, int dir, int* launches);

/*
 * p3_ftran_r2c_noalloc -- the forward transform of p3_ftran_r2c, but with the
 * workspace taken from a fixed device array built into the library instead
 * of from the caller.  The paper has no counterpart: this exists for callers
 * that must not allocate device memory when they run a transform (an
 * application that hands out all device memory from its own pre-sized pool
 * and forbids libraries to call cudaMalloc, or a latency-bound loop that
 * cannot afford a cudaMalloc/cudaFree, which can synchronise the device).
 * This call allocates nothing; the plan (created beforehand, which allocates
 * its small tables once) and the input / output buffers are the caller's.
 *   - The array holds P3_NOALLOC_SCRATCH_BYTES bytes per device, for as long
 *     as the process runs, on every GPU that loads the library.  Plans whose
 *     p3_plan_workspace_bytes() exceeds it get P3_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture begins.
 *   - All calls share the one array and it keeps the last call's contents
 *     (the transform overwrites every workspace element before reading it,
 *     so nothing needs clearing).  Calls whose kernels overlap on the GPU --
 *     on different streams, or from different threads -- race on it.
 *   - Errors as p3_ftran_r2c, plus P3_ERR_UNSUPPORTED for the size limit
 *     and for devices numbered 64 or higher (the per-device address table
 *     has 64 entries).
 */
#define P3_NOALLOC_SCRATCH_BYTES (64u << 20)
p3_status p3_ftran_r2c_noalloc(p3_plan plan, const void* in_real, void* out_cplx, void* stream);

/* Static string for a status code; never NULL. */
const char* p3_status_string(p3_status s);

/* P3_VERSION of the built library. */
int p3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* P3DFFT_GB300_H */
