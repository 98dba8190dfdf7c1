// lll_expand_host.cpp -- lll_simulate(LLL_EXPAND1 / LLL_EXPAND2): tables of
// the drift expansions (Eq. (drifta), Eq. (drifta2)) and the launch of
// expand_kernel (lll_expand.cu).
//
// The tables use the jump cumulant of the NIG driver in closed form,
//   kappa(u) = int (e^{ux} - 1 - ux) nu(dx)
//            = dbar (gamma - sqrt(alpha^2 - (beta + u)^2)) - u dbar beta / gamma,
// (the NIG cumulant of Section 4 with its mean removed), so the expansions
// need no quadrature nodes.  They are built in FP64 per Euler step for the
// live rates and stored in FP32.
#include <cmath>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lll.h"
#include "lll_ctx.h"
#include "lll_internal.h"

namespace lll {

int expand_threads();
size_t expand_smem(int order, int n, int ns);
int expand_occupancy(int order, size_t smem, int *blocks_per_sm);
int launch_expand(int order, int grid, size_t smem, cudaStream_t st, const PathArgs &a, const float *K1,
                  const float *K2, const float *K3);
int launch_finalize(const double *partials, int grid, int n_out, double *sums, cudaStream_t st);

namespace {

int build_tables(lll_ctx *ctx, int order)
{
    const int n = ctx->n, s = ctx->s, S = ctx->S;
    const double al = ctx->nig.alpha, be = ctx->nig.beta, db = ctx->nig.delta, ga = ctx->gam;
    bool domain_ok = true;
    auto kap = [&](double u) {
        const double r = al * al - (be + u) * (be + u);
        if (!(r > 0)) { domain_ok = false; return 0.0; }
        return db * (ga - std::sqrt(r)) - u * db * be / ga;
    };
    const size_t n2 = (size_t)n * n, n3 = n2 * n;
    std::vector<float> K1((size_t)S * n, 0.0f), K2((size_t)S * n2, 0.0f), K3;
    if (order == 2) K3.assign((size_t)S * n3, 0.0f);
    std::vector<double> k1(n), p2(n2);
    for (int k = 0; k < S; ++k) {
        const int imin = k / s + 1;
        const double *lam = ctx->lam.data() + (size_t)k * n;
        for (int i = imin; i <= n; ++i) k1[i - 1] = kap(lam[i - 1]);
        for (int i = imin; i <= n; ++i)
            for (int l = i + 1; l <= n; ++l) p2[(size_t)(i - 1) * n + (l - 1)] = kap(lam[i - 1] + lam[l - 1]);
        for (int i = imin; i <= n; ++i) {
            K1[(size_t)k * n + (i - 1)] = (float)k1[i - 1];
            for (int l = i + 1; l <= n; ++l)
                K2[(size_t)k * n2 + (size_t)(i - 1) * n + (l - 1)] =
                    (float)(p2[(size_t)(i - 1) * n + (l - 1)] - k1[i - 1] - k1[l - 1]);
            if (order == 2)
                for (int kk = i + 1; kk <= n; ++kk)
                    for (int l = kk + 1; l <= n; ++l) {
                        const double t3 = kap(lam[i - 1] + lam[kk - 1] + lam[l - 1]);
                        const double v = t3 - p2[(size_t)(i - 1) * n + (l - 1)] - p2[(size_t)(i - 1) * n + (kk - 1)] -
                                         p2[(size_t)(kk - 1) * n + (l - 1)] + k1[i - 1] + k1[kk - 1] + k1[l - 1];
                        K3[(size_t)k * n3 + (size_t)(i - 1) * n2 + (size_t)(kk - 1) * n + (l - 1)] = (float)v;
                    }
        }
    }
    if (!domain_ok)
        return record_error(ctx, LLL_EDOMAIN, "an expansion needs kappa at a sum of volatilities outside |beta + u| < alpha");
    float **dst[3] = {&ctx->d_K1, &ctx->d_K2, &ctx->d_K3};
    const std::vector<float> *src[3] = {&K1, &K2, &K3};
    for (int t = 0; t < 3; ++t) {
        cudaFree(*dst[t]);
        *dst[t] = nullptr;
        if (src[t]->empty()) continue;
        if (cudaMalloc((void **)dst[t], sizeof(float) * src[t]->size()) != cudaSuccess)
            return record_error(ctx, LLL_ENOMEM, "expansion tables");
        if (cudaMemcpy(*dst[t], src[t]->data(), sizeof(float) * src[t]->size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return record_error(ctx, LLL_ECUDA, "expansion tables upload");
    }
    ctx->expand_order = order;
    return LLL_OK;
}

}  // namespace

int simulate_expand(lll_ctx *ctx, int order, uint64_t first_path, uint64_t paths, uint64_t seed)
{
    if (ctx->driver != LLL_DRIVER_NIG)
        return record_error(ctx, LLL_EUNSUPPORTED, "drift expansions apply to the NIG driver's jump compensator");
    if ((order == 2 && ctx->n > 16) || ctx->n > 64)
        return record_error(ctx, LLL_EUNSUPPORTED, "drift expansions: n <= 16 rates (second order), n <= 64 (first)");
    LaunchPlan plan;
    int rc = plan_launch(ctx, LLL_FULL, first_path, paths, seed, &plan, false);
    if (rc != LLL_OK) return rc;
    if (ctx->expand_order != order) {
        rc = build_tables(ctx, order);
        if (rc != LLL_OK) return rc;
    }
    const int T = expand_threads();
    const size_t smem = expand_smem(order, ctx->n, ctx->ns);
    if (smem > 227 * 1024) return record_error(ctx, LLL_EUNSUPPORTED, "expansion tables exceed shared memory");
    int occ = 0;
    cudaError_t e = (cudaError_t)expand_occupancy(order, smem, &occ);
    if (e != cudaSuccess) return record_error(ctx, LLL_ECUDA, cudaGetErrorString(e));
    if (occ < 1) return record_error(ctx, LLL_EUNSUPPORTED, "expansion kernel does not fit on an SM");
    const uint64_t tiles = (paths + T - 1) / T;
    const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)occ * ctx->sm_count);
    const size_t state_need = (size_t)grid * ctx->n * T;
    if (state_need > ctx->state_cap) {
        cudaFree(ctx->d_state);
        ctx->d_state = nullptr;
        ctx->state_cap = 0;
        if (cudaMalloc((void **)&ctx->d_state, 4 * state_need) != cudaSuccess)
            return record_error(ctx, LLL_ENOMEM, "state scratch");
        ctx->state_cap = state_need;
    }
    const size_t nout = (size_t)plan.n_out;
    if ((size_t)grid * nout > ctx->partials_cap) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        if (cudaMalloc((void **)&ctx->d_partials, 8 * grid * nout) != cudaSuccess)
            return record_error(ctx, LLL_ENOMEM, "partials");
        ctx->partials_cap = (size_t)grid * nout;
    }
    if (nout > ctx->sums_cap) {
        cudaFree(ctx->d_sums);
        ctx->d_sums = nullptr;
        ctx->sums_cap = 0;
        if (cudaMalloc((void **)&ctx->d_sums, 8 * nout) != cudaSuccess) return record_error(ctx, LLL_ENOMEM, "sums");
        ctx->sums_cap = nout;
    }
    PathArgs a = plan.args;
    a.state = ctx->d_state;
    a.partials = ctx->d_partials;
    a.snap = ctx->d_snap; a.snap_stride = ctx->snap_stride; a.snap_pitch = ctx->n_snap;
    a.n_snap = ctx->d_snap ? std::min<uint64_t>(ctx->n_snap, (paths + ctx->snap_stride - 1) / ctx->snap_stride) : 0;
    cudaStream_t st = ctx->stream;
#define XTRY(expr)                                                                                 \
    do {                                                                                           \
        cudaError_t e2 = (cudaError_t)(expr);                                                      \
        if (e2 != cudaSuccess) return record_error(ctx, LLL_ECUDA, cudaGetErrorString(e2));       \
    } while (0)
    XTRY(cudaEventRecord(ctx->ev[0], st));
    XTRY(launch_expand(order, grid, smem, st, a, ctx->d_K1, ctx->d_K2, ctx->d_K3));
    XTRY(cudaEventRecord(ctx->ev[1], st));
    XTRY(launch_finalize(ctx->d_partials, grid, (int)nout, ctx->d_sums, st));
    XTRY(cudaEventRecord(ctx->ev[2], st));
#undef XTRY
    ctx->simulated = true;
    ctx->err_pending = false;
    ctx->gemm_err_pending = false;
    ctx->last_paths = paths;
    ctx->last_snap_paths = a.n_snap;
    return LLL_OK;
}

}  // namespace lll
