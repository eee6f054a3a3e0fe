// Configuration, set-up and launch of the power-of-two stage kernels
// (templates in p3_pow2.cuh, instantiated per precision in p3_pow2_f32.cu and
// p3_pow2_f64.cu).
#include <cudaTypedefs.h>

#include "p3_internal.h"

namespace p3 {

void* pow2_pick_f32(int kind, int N, bool inv, int sym);
void* pow2_pick_f64(int kind, int N, bool inv, int sym);
void pow2_shape_f32(int kind, int N, int* B, int* tpl, size_t* smem);
void pow2_shape_f64(int kind, int N, int* B, int* tpl, size_t* smem);

void* pow2_pick_tma_f32(int N, int sym);
size_t pow2_tma_smem_f32(int N, int sym);
void* pow2_pick_zbulk_f32(int N);
size_t pow2_zbulk_smem_f32(int N);

// Column-kernel symmetry variant of a stage: 0 plain, 1 DCT-I, 2 DST-I.
static int sym_of(const StageArgs& a) { return a.op == OP_DCT1 ? 1 : a.op == OP_DST1 ? 2 : 0; }

namespace {
bool is_pow2_in_range(int n) { return n >= 64 && n <= 4096 && (n & (n - 1)) == 0; }
}  // namespace

static bool configure(StageArgs& a, size_t csize, bool allow_tma);

bool pow2_configure(StageArgs& a, size_t csize, bool allow_tma)
{
    StageArgs b = a;  // a keeps its generic configuration unless this succeeds
    if (!configure(b, csize, allow_tma)) return false;
    a = b;
    return true;
}

static bool configure(StageArgs& a, size_t csize, bool allow_tma)
{
    if (a.blue) return false;
    const int N = a.nfft;
    if (!is_pow2_in_range(N)) return false;
    const bool f32 = csize == 8;
    int kind = 0;
    if (a.op == OP_C2C || a.op == OP_DCT1 || a.op == OP_DST1) {
        const bool in_adj = a.in.lstride == 1, out_adj = a.out.lstride == 1;
        const bool in_el = a.in.es == 1, out_el = a.out.es == 1;
        if (in_adj && out_adj && !in_el && !out_el) kind = KIND_COL_DD;
        else if (in_adj && !in_el && out_el) kind = KIND_COL_DS;
        else if (in_el && out_adj && !out_el) kind = KIND_COL_SD;
        else return false;
    } else if (a.op == OP_R2C_HALF || a.op == OP_C2R_HALF) {
        if (a.in.es != 1 || a.out.es != 1) return false;
        kind = a.op == OP_R2C_HALF ? KIND_ROW_R2C : KIND_ROW_C2R;
    } else {
        return false;
    }
    int B = 1, tpl = 1;
    size_t smem = 0;
    if (f32) pow2_shape_f32(kind, N, &B, &tpl, &smem);
    else pow2_shape_f64(kind, N, &B, &tpl, &smem);
    a.B = B;
    a.LDB = B;
    a.tpl = tpl;
    a.threads = B * tpl;
    a.smem = smem;
    a.kern = kind;
    a.tma = 0;
    // TMA-staged input tile for the forward ZYX store: the tile's lines must
    // be adjacent (the tensor's inner dimension) and their elements a
    // 16-byte multiple apart, past the last line
    if (f32 && allow_tma && kind == KIND_COL_DS && N >= 256 && N <= 2048 && a.in.lstride == 1 &&
        a.in.per >= a.nlines && a.in.es % 2 == 0 && a.in.es >= a.nlines && (B % 2) == 0) {
        a.tma = 1;
        a.smem = pow2_tma_smem_f32(N, sym_of(a));
    }
    // bulk-copied tile for the row-style ZYX load: plain FFT lines that lie
    // one after another in memory
    if (f32 && allow_tma && kind == KIND_COL_SD && a.op == OP_C2C && a.sign > 0 && a.n_in == N &&
        a.in.es == 1 && a.in.lstride == N && a.in.per >= a.nlines && pow2_pick_zbulk_f32(N)) {
        a.tma = 2;
        a.smem = pow2_zbulk_smem_f32(N);
    }
    return true;
}

cudaError_t pow2_prepare()
{
    for (int f = 0; f < 2; ++f)
        for (int kind = KIND_COL_DD; kind <= KIND_ROW_C2R; ++kind)
            for (int N = 64; N <= 4096; N *= 2)
                for (int inv = 0; inv < 2; ++inv)
                    for (int sym = 0; sym < 3; ++sym) {
                            void* fn = f == 0 ? pow2_pick_f32(kind, N, inv, sym) : pow2_pick_f64(kind, N, inv, sym);
                            if (f == 0 && kind == KIND_COL_SD && inv && sym == 0) {
                                void* fb = pow2_pick_zbulk_f32(N);
                                if (fb && cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               227 * 1024) != cudaSuccess)
                                    return cudaGetLastError();
                            }
                            if (f == 0 && kind == KIND_COL_DS && !inv) {
                                void* ft = pow2_pick_tma_f32(N, sym);
                                if (ft && cudaFuncSetAttribute(ft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               227 * 1024) != cudaSuccess)
                                    return cudaGetLastError();
                            }
                            if (!fn) continue;
                            cudaError_t e =
                                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
                            if (e != cudaSuccess) return e;
                        }
    return cudaSuccess;
}

cudaError_t pow2_launch(const StageArgs& a, bool f32, cudaStream_t st)
{
    const bool inv = a.sign > 0;
    const int sym = sym_of(a);
    void* fn = a.tma == 2 ? pow2_pick_zbulk_f32(a.nfft)
               : a.tma ? pow2_pick_tma_f32(a.nfft, sym)
                     : (f32 ? pow2_pick_f32(a.kern, a.nfft, inv, sym) : pow2_pick_f64(a.kern, a.nfft, inv, sym));
    if (!fn) return cudaErrorInvalidDeviceFunction;
    if (a.nlines <= 0) return cudaSuccess;
    long long grid = (a.nlines + a.B - 1) / a.B;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    StageArgs m = a;
    line_magic(m.in, m.nlines);
    line_magic(m.out, m.nlines);
    void* args[] = {&m};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(m.threads), args, m.smem, st);
}

// cuTensorMapEncodeTiled, from the driver through the runtime (resolved once)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

cudaError_t pow2_encode_tma(StageArgs& a)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // 8-byte complex elements: lines (inner, unit stride) x line elements (outer, es apart)
    const cuuint64_t dims[2] = {(cuuint64_t)a.nlines, (cuuint64_t)a.n_in};
    const cuuint64_t strides[1] = {(cuuint64_t)a.in.es * 8};
    const cuuint32_t box[2] = {(cuuint32_t)a.B, 256};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(a.src), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace p3
