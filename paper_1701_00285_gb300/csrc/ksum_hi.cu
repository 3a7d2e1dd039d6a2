// Kernel sums for point dimensions 9..16 (the kernels live in ksum_impl.cuh;
// instantiated here so that they compile beside the d <= 8 ones).
#include "ksum_impl.cuh"

namespace mlb {

bool kernel_sum_hi(mlb_ctx* ctx, const double* tg, int64_t M, const double* sources, int64_t Ns,
                   const double* weights, double* out, const TrendArgs& tr, bool deriv, bool accurate) {
    switch (ctx->d) {
#define MLB_KSUM_CASE(DD)                                                                     \
    case DD:                                                                                  \
        if (deriv) launch_ksum<DD, true>(ctx, tg, M, sources, Ns, weights, out, tr, accurate); \
        else launch_ksum<DD, false>(ctx, tg, M, sources, Ns, weights, out, tr, accurate);      \
        return true;
        MLB_KSUM_CASE(9) MLB_KSUM_CASE(10) MLB_KSUM_CASE(11) MLB_KSUM_CASE(12)
        MLB_KSUM_CASE(13) MLB_KSUM_CASE(14) MLB_KSUM_CASE(15) MLB_KSUM_CASE(16)
#undef MLB_KSUM_CASE
        default: return false;
    }
}

}  // namespace mlb
