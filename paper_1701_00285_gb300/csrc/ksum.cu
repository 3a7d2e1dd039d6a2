// Kernel sums: dispatch for d <= 8, the launch-shape autotuner and the entry
// points used by the other files (kernels in ksum_impl.cuh; d >= 9 in ksum_hi.cu).
#include "ksum_impl.cuh"

namespace mlb {

bool kernel_sum_hi(mlb_ctx* ctx, const double* tg, int64_t M, const double* sources, int64_t Ns,
                   const double* weights, double* out, const TrendArgs& tr, bool deriv, bool accurate);

mlb_status kernel_sum_general(mlb_ctx* ctx, const double* targets, int64_t M, const double* sources, int64_t Ns,
                              const double* weights, double* out, bool add_trend, bool deriv, bool accurate) {
    if (M <= 0) return MLB_OK;
    TrendArgs tr{};
    tr.beta = add_trend ? ctx->beta : nullptr;
    tr.alpha = ctx->alpha;
    tr.p = ctx->p;
    for (int c = 0; c < ctx->d; ++c) {
        tr.lo[c] = ctx->box_lo[c];
        tr.hi[c] = ctx->box_hi[c];
    }
    const double* tg = targets ? targets : ctx->xs;
    if (!sources) Ns = ctx->N;
    // the matrix-free product's sum of the data points against themselves:
    // the tensor-core form when the autotuner chose it
    if (ctx->ksum_variant == kKsumVariantTC && ctx->opts.precision == MLB_MIXED && !accurate && !deriv &&
        !targets && !sources && !add_trend && M == ctx->N && ksum_tc_self(ctx, weights, out))
        return MLB_OK;
    switch (ctx->d) {
#define MLB_KSUM_CASE(DD)                                                                          \
    case DD:                                                                                       \
        if (deriv) launch_ksum<DD, true>(ctx, tg, M, sources, Ns, weights, out, tr, accurate);   \
        else launch_ksum<DD, false>(ctx, tg, M, sources, Ns, weights, out, tr, accurate);        \
        break;
        MLB_KSUM_CASE(1) MLB_KSUM_CASE(2) MLB_KSUM_CASE(3) MLB_KSUM_CASE(4)
        MLB_KSUM_CASE(5) MLB_KSUM_CASE(6) MLB_KSUM_CASE(7) MLB_KSUM_CASE(8)
#undef MLB_KSUM_CASE
        default:
            if (ctx->d > kMaxDim || !kernel_sum_hi(ctx, tg, M, sources, Ns, weights, out, tr, deriv, accurate))
                return fail(ctx, MLB_EINVAL, "dimension d out of range 1..16");
    }
    MLB_CHECK_LAUNCH(ctx, "kernel sum");
    return MLB_OK;
}

// Autotuner for the FP32 kernel sum of the matrix-free product: times every
// launch shape, and the tensor-core form where the dimension and covariance
// have one, once on the context's own points (CUDA events on its stream) and
// keeps the fastest, cached per (device, dimension, covariance kind,
// problem-size bucket) for the rest of the process.  Runs outside any stream
// capture.
static std::mutex g_tune_mutex;
static std::map<std::tuple<int, int, int, int>, int> g_tune_cache;

mlb_status tune_kernel_sum(mlb_ctx* ctx) {
    ctx->ksum_variant = 1;
    if (ctx->opts.precision != MLB_MIXED) return MLB_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    int bucket = 0;
    while ((1LL << (bucket + 1)) <= ctx->N) ++bucket;
    const auto key = std::make_tuple(dev, ctx->d, ctx->kfn.kind, bucket);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            ctx->ksum_variant = it->second;
            return MLB_OK;
        }
    }
    double* a = ctx->vec + 8 * ctx->N;
    double* b = ctx->vec + 9 * ctx->N;
    MLB_CUDA(ctx, cudaMemsetAsync(a, 0, sizeof(double) * ctx->N, ctx->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bestv = 1;
    for (int v = 0; v <= kKsumVariantTC; ++v) {
        if (v == kKsumVariantTC && !ksum_tc_supported(ctx)) continue;
        ctx->ksum_variant = v;
        mlb_status s = kernel_sum_general(ctx, nullptr, ctx->N, nullptr, ctx->N, a, b, false, false, false);
        if (s != MLB_OK) break;
        cudaEventRecord(e0, ctx->stream);
        s = kernel_sum_general(ctx, nullptr, ctx->N, nullptr, ctx->N, a, b, false, false, false);
        cudaEventRecord(e1, ctx->stream);
        if (s != MLB_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bestv = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->ksum_variant = bestv;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = bestv;
    return MLB_OK;
}

mlb_status kernel_sum_dev(mlb_ctx* ctx, const double* targets, int64_t M, const double* a_kd, double* out,
                          bool add_trend) {
    return kernel_sum_general(ctx, targets, M, nullptr, ctx->N, a_kd, out, add_trend, false);
}

}  // namespace mlb
