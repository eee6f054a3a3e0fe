// Instantiations of the power-of-two stage kernels for float data.
#include "p3_pow2.cuh"

namespace p3 {

namespace {
using namespace pw;

template <int N, int MODE, bool INV, bool DCT> void* col_fn()
{
    return (void*)col_kernel<float, N, col_E<float>(N, MODE), col_B<float>(N), MODE, INV, DCT>;
}
template <int N, int MODE, bool INV, bool DCT> void* col_pl_fn()
{
    if constexpr (col_pipelined<float>(N, MODE))
        return (void*)col_kernel_pl<float, N, col_pl_E<float>(N, MODE), col_B<float>(N), MODE, INV, DCT>;
    else
        return nullptr;
}
template <int N, int OPR> void* row_fn() { return (void*)row_kernel<float, N, row_E<float>(N), row_B<float>(N), OPR>; }

#define P3_COL_PICK(FN, MODE) \
    (inv ? (dct ? FN<N, MODE, true, true>() : FN<N, MODE, true, false>()) \
         : (dct ? FN<N, MODE, false, true>() : FN<N, MODE, false, false>()))
template <int N> void* pick_n(int kind, bool inv, bool dct, bool pl)
{
    switch (kind) {
    case KIND_COL_DD: return pl ? P3_COL_PICK(col_pl_fn, 0) : P3_COL_PICK(col_fn, 0);
    case KIND_COL_DS: return pl ? P3_COL_PICK(col_pl_fn, 1) : P3_COL_PICK(col_fn, 1);
    case KIND_COL_SD: return pl ? P3_COL_PICK(col_pl_fn, 2) : P3_COL_PICK(col_fn, 2);
    case KIND_ROW_R2C: return pl ? nullptr : row_fn<N, 0>();
    case KIND_ROW_C2R: return pl ? nullptr : row_fn<N, 1>();
    default: return nullptr;
    }
}
#undef P3_COL_PICK
}  // namespace

void* pow2_pick_f32(int kind, int N, bool inv, bool dct, bool pl)
{
    switch (N) {
    case 64: return pick_n<64>(kind, inv, dct, pl);
    case 128: return pick_n<128>(kind, inv, dct, pl);
    case 256: return pick_n<256>(kind, inv, dct, pl);
    case 512: return pick_n<512>(kind, inv, dct, pl);
    case 1024: return pick_n<1024>(kind, inv, dct, pl);
    case 2048: return pick_n<2048>(kind, inv, dct, pl);
    case 4096: return pick_n<4096>(kind, inv, dct, pl);
    default: return nullptr;
    }
}

void pow2_shape_f32(int kind, int N, int* B, int* tpl, size_t* smem, int* pl)
{
    using namespace pw;
    *pl = 0;
    if (kind == KIND_ROW_R2C || kind == KIND_ROW_C2R) {
        const int E = row_E<float>(N);
        *B = row_B<float>(N);
        *tpl = N / E;
        *smem = (size_t)(*B) * (size_t)(N + N / E + 1) * sizeof(float) * 2;
    } else {
        const int mode = kind == KIND_COL_SD ? 2 : kind == KIND_COL_DS ? 1 : 0;
        *B = col_B<float>(N);
        const size_t slots = (size_t)(cpad_c(N - 1) + 1) * (size_t)(*B);
        if (col_pipelined<float>(N, mode)) {
            *pl = 1;
            *tpl = N / col_pl_E<float>(N, mode);
            *smem = 2 * slots * sizeof(float) * 2;
        } else {
            *tpl = N / col_E<float>(N, mode);
            *smem = slots * sizeof(float) * 2;
        }
    }
}

}  // namespace p3
