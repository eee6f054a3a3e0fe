// Instantiations of the power-of-two stage kernels for float data.
#include "p3_pow2.cuh"

namespace p3 {

namespace {
using namespace pw;

template <int N, int MODE, bool INV, int SYM> void* col_fn()
{
    return (void*)col_kernel<float, N, col_E<float>(N, MODE), col_B<float>(N), MODE, INV, SYM>;
}
template <int N, bool INV, int SYM> void* zrow_fn()
{
    if constexpr (col_zrow<float>(N))
        return (void*)zrow_kernel<float, N, row_E<float>(N), zrow_B<float>(N), INV, SYM>;
    else
        return nullptr;
}
template <int N, int SYM> void* tma_fn()
{
    return (void*)col_kernel_tma<float, N, col_E<float>(N, 1), col_B<float>(N), SYM>;
}
template <int N, int OPR> void* row_fn() { return (void*)row_kernel<float, N, row_E<float>(N), row_B<float>(N), OPR>; }

// sym: 0 plain, 1 Chebyshev (DCT-I), 2 sine (DST-I, forward sign only)
#define P3_COL_PICK(FN, MODE) \
    (sym == 2 ? (inv ? (void*)nullptr : FN<N, MODE, false, 2>()) \
     : inv ? (sym ? FN<N, MODE, true, 1>() : FN<N, MODE, true, 0>()) \
           : (sym ? FN<N, MODE, false, 1>() : FN<N, MODE, false, 0>()))
template <int N> void* pick_n(int kind, bool inv, int sym)
{
    switch (kind) {
    case KIND_COL_DD: return P3_COL_PICK(col_fn, 0);
    case KIND_COL_DS: return P3_COL_PICK(col_fn, 1);
    case KIND_COL_SD:
        if (col_zrow<float>(N))
            return sym == 2 ? (inv ? (void*)nullptr : zrow_fn<N, false, 2>())
                   : inv ? (sym ? zrow_fn<N, true, 1>() : zrow_fn<N, true, 0>())
                         : (sym ? zrow_fn<N, false, 1>() : zrow_fn<N, false, 0>());
        return P3_COL_PICK(col_fn, 2);
    case KIND_ROW_R2C: return row_fn<N, 0>();
    case KIND_ROW_C2R: return row_fn<N, 1>();
    default: return nullptr;
    }
}
#undef P3_COL_PICK
}  // namespace

void* pow2_pick_f32(int kind, int N, bool inv, int sym)
{
    switch (N) {
    case 64: return pick_n<64>(kind, inv, sym);
    case 128: return pick_n<128>(kind, inv, sym);
    case 256: return pick_n<256>(kind, inv, sym);
    case 512: return pick_n<512>(kind, inv, sym);
    case 1024: return pick_n<1024>(kind, inv, sym);
    case 2048: return pick_n<2048>(kind, inv, sym);
    case 4096: return pick_n<4096>(kind, inv, sym);
    default: return nullptr;
    }
}

// Row-style ZYX-load kernels with a bulk-copied input tile (FP32 plain FFT lines, 256 .. 1024 points)
void* pow2_pick_zbulk_f32(int N)
{
    switch (N) {
    case 256: return (void*)zrow_kernel<float, 256, row_E<float>(256), row_B<float>(256), true, 0, true>;
    case 512: return (void*)zrow_kernel<float, 512, row_E<float>(512), row_B<float>(512), true, 0, true>;
    case 1024: return (void*)zrow_kernel<float, 1024, row_E<float>(1024), row_B<float>(1024), true, 0, true>;
    case 2048: return (void*)zrow_kernel<float, 2048, row_E<float>(2048), zrow_B<float>(2048), true, 0, true>;
    default: return nullptr;
    }
}
size_t pow2_zbulk_smem_f32(int N)
{
    using namespace pw;
    switch (N) {
    case 256: return zrow_bulk_smem<float, 256, row_E<float>(256), row_B<float>(256)>();
    case 512: return zrow_bulk_smem<float, 512, row_E<float>(512), row_B<float>(512)>();
    case 1024: return zrow_bulk_smem<float, 1024, row_E<float>(1024), row_B<float>(1024)>();
    case 2048: return zrow_bulk_smem<float, 2048, row_E<float>(2048), zrow_B<float>(2048)>();
    default: return 0;
    }
}

// TMA-staged ZYX-store kernels (FP32, 256 .. 2048 points): kernel and dynamic shared memory
void* pow2_pick_tma_f32(int N, int sym)
{
    switch (N) {
    case 256: return sym == 2 ? tma_fn<256, 2>() : sym ? tma_fn<256, 1>() : tma_fn<256, 0>();
    case 512: return sym == 2 ? tma_fn<512, 2>() : sym ? tma_fn<512, 1>() : tma_fn<512, 0>();
    case 1024: return sym == 2 ? tma_fn<1024, 2>() : sym ? tma_fn<1024, 1>() : tma_fn<1024, 0>();
    case 2048: return sym == 2 ? tma_fn<2048, 2>() : sym ? tma_fn<2048, 1>() : tma_fn<2048, 0>();
    default: return nullptr;
    }
}
size_t pow2_tma_smem_f32(int N, int sym)
{
    using namespace pw;
    switch (N) {
    case 256: return col_tma_smem<float, 256, col_B<float>(256)>(sym);
    case 512: return col_tma_smem<float, 512, col_B<float>(512)>(sym);
    case 1024: return col_tma_smem<float, 1024, col_B<float>(1024)>(sym);
    case 2048: return col_tma_smem<float, 2048, col_B<float>(2048)>(sym);
    default: return 0;
    }
}

void pow2_shape_f32(int kind, int N, int* B, int* tpl, size_t* smem)
{
    using namespace pw;
    if (kind == KIND_ROW_R2C || kind == KIND_ROW_C2R) {
        const int E = row_E<float>(N);
        *B = row_B<float>(N);
        *tpl = N / E;
        *smem = (size_t)(*B) * (size_t)(N + N / E + 1) * sizeof(float) * 2;
    } else if (kind == KIND_COL_SD && col_zrow<float>(N)) {
        const int E = row_E<float>(N);
        *B = zrow_B<float>(N);
        *tpl = N / E;
        switch (N) {
        case 256: *smem = zrow_smem<float, 256, row_E<float>(256), zrow_B<float>(256)>(); break;
        case 512: *smem = zrow_smem<float, 512, row_E<float>(512), zrow_B<float>(512)>(); break;
        case 1024: *smem = zrow_smem<float, 1024, row_E<float>(1024), zrow_B<float>(1024)>(); break;
        default: *smem = zrow_smem<float, 2048, row_E<float>(2048), zrow_B<float>(2048)>(); break;
        }
    } else {
        const int mode = kind == KIND_COL_SD ? 2 : kind == KIND_COL_DS ? 1 : 0;
        *B = col_B<float>(N);
        const size_t slots = (size_t)(cpad_c(N - 1) + 1) * (size_t)(*B);
        *tpl = N / col_E<float>(N, mode);
        *smem = slots * sizeof(float) * 2;
    }
}

}  // namespace p3
