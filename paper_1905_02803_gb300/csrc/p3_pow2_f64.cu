// Instantiations of the power-of-two stage kernels for double data.
#include "p3_pow2.cuh"

namespace p3 {

namespace {
using namespace pw;

template <int N, int MODE, bool INV, bool DCT> void* col_fn()
{
    return (void*)col_kernel<double, N, col_E<double>(N, MODE), col_B<double>(N), MODE, INV, DCT>;
}
template <int N, int OPR> void* row_fn() { return (void*)row_kernel<double, N, row_E<double>(N), row_B<double>(N), OPR>; }

template <int N> void* pick_n(int kind, bool inv, bool dct)
{
    switch (kind) {
    case KIND_COL_DD:
        return inv ? (dct ? col_fn<N, 0, true, true>() : col_fn<N, 0, true, false>())
                   : (dct ? col_fn<N, 0, false, true>() : col_fn<N, 0, false, false>());
    case KIND_COL_DS:
        return inv ? (dct ? col_fn<N, 1, true, true>() : col_fn<N, 1, true, false>())
                   : (dct ? col_fn<N, 1, false, true>() : col_fn<N, 1, false, false>());
    case KIND_COL_SD:
        return inv ? (dct ? col_fn<N, 2, true, true>() : col_fn<N, 2, true, false>())
                   : (dct ? col_fn<N, 2, false, true>() : col_fn<N, 2, false, false>());
    case KIND_ROW_R2C: return row_fn<N, 0>();
    case KIND_ROW_C2R: return row_fn<N, 1>();
    default: return nullptr;
    }
}
}  // namespace

void* pow2_pick_f64(int kind, int N, bool inv, bool dct)
{
    switch (N) {
    case 64: return pick_n<64>(kind, inv, dct);
    case 128: return pick_n<128>(kind, inv, dct);
    case 256: return pick_n<256>(kind, inv, dct);
    case 512: return pick_n<512>(kind, inv, dct);
    case 1024: return pick_n<1024>(kind, inv, dct);
    case 2048: return pick_n<2048>(kind, inv, dct);
    case 4096: return pick_n<4096>(kind, inv, dct);
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
    } else {
        const int E = col_E<double>(N, kind == KIND_COL_SD ? 2 : kind == KIND_COL_DS ? 1 : 0);
        *B = col_B<double>(N);
        *tpl = N / E;
        *smem = (size_t)(cpad_c(N - 1) + 1) * (size_t)(*B) * sizeof(double) * 2;
    }
}

}  // namespace p3
