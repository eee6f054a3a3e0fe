// Instantiations of the power-of-two stage kernels for double data.
#include "p3_pow2.cuh"

namespace p3 {

namespace {
using namespace pw;

template <int N, int MODE, bool INV, int SYM> void* col_fn()
{
    return (void*)col_kernel<double, N, col_E<double>(N, MODE), col_B<double>(N), MODE, INV, SYM>;
}
template <int N, bool INV, int SYM> void* zrow_fn()
{
    if constexpr (col_zrow<double>(N))
        return (void*)zrow_kernel<double, N, row_E<double>(N), zrow_B<double>(N), INV, SYM>;
    else
        return nullptr;
}
template <int N, int OPR> void* row_fn() { return (void*)row_kernel<double, N, row_E<double>(N), row_B<double>(N), OPR>; }

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
        if (col_zrow<double>(N))
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

void* pow2_pick_f64(int kind, int N, bool inv, int sym)
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

void pow2_shape_f64(int kind, int N, int* B, int* tpl, size_t* smem)
{
    using namespace pw;
    if (kind == KIND_ROW_R2C || kind == KIND_ROW_C2R) {
        const int E = row_E<double>(N);
        *B = row_B<double>(N);
        *tpl = N / E;
        *smem = (size_t)(*B) * (size_t)(N + N / E + 1) * sizeof(double) * 2;
    } else if (kind == KIND_COL_SD && col_zrow<double>(N)) {
        const int E = row_E<double>(N);
        *B = row_B<double>(N);
        *tpl = N / E;
        switch (N) {
        case 256: *smem = zrow_smem<double, 256, row_E<double>(256), row_B<double>(256)>(); break;
        case 512: *smem = zrow_smem<double, 512, row_E<double>(512), row_B<double>(512)>(); break;
        default: *smem = zrow_smem<double, 1024, row_E<double>(1024), row_B<double>(1024)>(); break;
        }
    } else {
        const int mode = kind == KIND_COL_SD ? 2 : kind == KIND_COL_DS ? 1 : 0;
        *B = col_B<double>(N);
        const size_t slots = (size_t)(cpad_c(N - 1) + 1) * (size_t)(*B);
        *tpl = N / col_E<double>(N, mode);
        *smem = slots * sizeof(double) * 2;
    }
}

}  // namespace p3
