// lll_capi.cpp -- the C ABI declared in include/lll.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lll.h"
#include "lll_ctx.h"
#include "lll_internal.h"

namespace lll {
int build_nig_rule(double alpha, double beta, double dbar, double a, int Q, double *nodes,
                   double *weights);
int simulate_mlp(lll_ctx *ctx, uint64_t first_path, uint64_t paths, uint64_t seed);
int simulate_expand(lll_ctx *ctx, int order, uint64_t first_path, uint64_t paths, uint64_t seed);
}

using namespace lll;

namespace {

thread_local std::string g_err;

int fail(lll_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    g_err = msg;
    return code;
}

int cuda_fail(lll_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, LLL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, expr)                                                                        \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);                                   \
    } while (0)

bool isfin(double v) { return std::isfinite(v); }

int padded_q(int Q)
{
    if (Q <= 0) return 0;
    const int opts[] = {16, 32, 64, 96, 128};
    for (int o : opts)
        if (Q <= o) return o;
    return -1;
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(count, 1));
}

void free_all(lll_ctx *c)
{
    cudaFree(c->d_lam); cudaFree(c->d_x); cudaFree(c->d_W); cudaFree(c->d_w0); cudaFree(c->d_b0);
    cudaFree(c->d_tab); cudaFree(c->d_row); cudaFree(c->d_Z0); cudaFree(c->d_c0);
    cudaFree(c->d_strikes); cudaFree(c->d_partials); cudaFree(c->d_sums); cudaFree(c->d_state);
    cudaFree(c->d_snap); cudaFree(c->d_C); cudaFree(c->d_cn); cudaFree(c->d_err);
    cudaFree(c->d_K1); cudaFree(c->d_K2); cudaFree(c->d_K3);
    mlp_free(c->mlp);
    c->mlp = nullptr;
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
}

int default_chunk_rows(int n, int QP)
{
    if (QP == 0) return std::min(n, 64);
    // Keep the double-buffered node tables near 24 KB (room for five blocks per SM).
    const int rows = (24 * 1024) / (2 * (QP / 4) * (int)sizeof(float4));
    return std::max(1, std::min(n, rows));
}

}  // namespace

namespace lll {

int record_error(lll_ctx *ctx, int code, const char *msg) { return fail(ctx, code, msg); }

int launch_plan(const LaunchPlan &plan, const PathArgs &a)
{
    if (plan.tenor > 0) return launch_tenor_kernel(plan.scheme, plan.qp, plan.tenor, plan.grid, plan.smem, plan.stream, a);
    if (plan.lpp > 1)
        return launch_group_kernel(plan.scheme, plan.qp, plan.lpp, plan.grid, plan.threads, plan.smem, plan.stream, a);
    return launch_path_kernel(plan.scheme, plan.qp, plan.ppt, plan.grid, plan.threads, plan.smem, plan.stream, a);
}

// Same launch shape and arguments as lll_simulate, with no allocation: the
// per-block scratch sizes are returned for the caller to place.
int plan_launch(lll_ctx *ctx, int scheme, uint64_t first_path, uint64_t paths, uint64_t seed,
                LaunchPlan *plan, bool allow_tenor)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (!plan) return fail(ctx, LLL_EINVAL, "plan is NULL");
    if (scheme == LLL_MLP || scheme == LLL_EXPAND1 || scheme == LLL_EXPAND2)
        return fail(ctx, LLL_EUNSUPPORTED, "LLL_MLP and LLL_EXPAND1/2 run through lll_simulate only");
    if (scheme != LLL_FULL && scheme != LLL_PICARD && scheme != LLL_FROZEN)
        return fail(ctx, LLL_EINVAL, "unknown scheme");
    if (ctx->ns == 0) return fail(ctx, LLL_ESTATE, "lll_set_strikes must come before simulating");
    if (paths == 0) return fail(ctx, LLL_EINVAL, "paths must be > 0");
    if (first_path + paths < first_path) return fail(ctx, LLL_EINVAL, "path range overflows");
    const int QPk = (scheme == LLL_FROZEN) ? 0 : ctx->QP;
    // Tenor-parallel mapping (lll_set_mapping): G lanes per path, full and
    // Picard with a node table and caplet payoffs; other schemes keep the
    // path mapping.
    const int G = (allow_tenor && ctx->tenor_lanes > 0 && (scheme == LLL_FULL || scheme == LLL_PICARD))
                      ? ctx->tenor_lanes : 0;
    if (G > 0) {
        if (QPk == 0 || ctx->product != LLL_PRODUCT_CAPLET || !tenor_kernel_supported(scheme, QPk, G))
            return fail(ctx, LLL_EUNSUPPORTED, "the tenor-parallel mapping needs a node table and caplet payoffs");
    }
    // Lanes per group of paths: 1 (one lane sweeps all nodes of its path) or
    // 2 / 4 (lane groups share the node sweep); the default is 1.
    const int lpp = G > 0 ? 1 : (ctx->lpp > 0 ? ctx->lpp : 1);
    const int R = (lpp > 1 || G > 0) ? 1 : (ctx->ppt > 0 ? ctx->ppt : 1);
    if (lpp > 1 && !group_kernel_supported(scheme, QPk, lpp))
        return fail(ctx, LLL_EUNSUPPORTED, "lane groups need a node table (NIG, full or Picard)");
    if (G == 0 && lpp == 1 && !path_kernel_supported(scheme, QPk, R))
        return fail(ctx, LLL_EUNSUPPORTED, "no kernel for this Q and paths per thread");
    const int T = G > 0 ? tenor_kernel_threads() : ctx->threads, CH = ctx->chunk_rows;
    const size_t smem = G > 0 ? tenor_kernel_smem(QPk, ctx->n, ctx->ns, G)
                      : lpp > 1 ? group_kernel_smem(QPk, ctx->n, ctx->ns, T, CH)
                                : path_kernel_smem(QPk, ctx->n, ctx->ns, T, CH);
    if (smem > 227 * 1024) return fail(ctx, LLL_EUNSUPPORTED, "shared memory need exceeds 227 KB");
    int occ = 0;
    cudaError_t e;
    if (G > 0) {
        e = (cudaError_t)tenor_kernel_prepare(scheme, QPk, G, smem, &occ);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tenor kernel attributes");
    } else if (lpp > 1) {
        e = (cudaError_t)group_kernel_prepare(scheme, QPk, lpp, smem, T, &occ);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "group kernel attributes");
    } else {
        e = (cudaError_t)path_kernel_prepare(scheme, QPk, R, T, smem);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
        e = (cudaError_t)path_kernel_occupancy(scheme, QPk, R, T, smem, &occ);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
    }
    if (occ < 1) return fail(ctx, LLL_EUNSUPPORTED, "launch shape does not fit on an SM");
    const int bps = ctx->blocks_per_sm > 0 ? std::min(ctx->blocks_per_sm, occ) : occ;
    const uint64_t per_tile = G > 0 ? (uint64_t)(T / G) : (uint64_t)T * R; // paths per block tile
    const uint64_t tiles = (paths + per_tile - 1) / per_tile;
    const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)bps * ctx->sm_count);
    const int nst = (scheme == LLL_PICARD) ? 2 : 1;
    PathArgs a{};
    a.tab = ctx->d_tab; a.cn = ctx->d_cn; a.row = ctx->d_row; a.Z0 = ctx->d_Z0; a.c0 = ctx->d_c0;
    a.strikes = ctx->d_strikes; a.partials = nullptr; a.state = nullptr;
    a.snap = nullptr; a.n_snap = 0; a.snap_stride = 1; a.snap_pitch = 0;
    a.first_path = first_path; a.paths = paths;
    a.n = ctx->n; a.s = ctx->s; a.S = ctx->S; a.ns = ctx->ns; a.chunk_rows = CH;
    a.key0 = (uint32_t)seed; a.key1 = (uint32_t)(seed >> 32); a.inst = 0;
    a.driver = ctx->driver;
    a.h = (float)ctx->h; a.sqrt_h = (float)std::sqrt(ctx->h); a.delta = (float)ctx->delta;
    a.dBN = (float)(ctx->delta * ctx->BN);
    a.product = ctx->product;
    if (ctx->driver == LLL_DRIVER_NIG) {
        const double m = ctx->nig.delta * ctx->h / ctx->gam;
        const double l = (ctx->nig.delta * ctx->h) * (ctx->nig.delta * ctx->h);
        a.ig_m = (float)m; a.ig_m2 = (float)(m * m); a.ig_hl = (float)(m / (2.0 * l));
        a.ig_fl = (float)(4.0 * m * l); a.ig_md = m; a.ig_ld = l;
        a.nig_beta = (float)ctx->nig.beta; a.nig_muh = (float)(ctx->mu * ctx->h);
    }
    plan->args = a;
    plan->scheme = scheme; plan->qp = QPk; plan->ppt = R; plan->lpp = lpp; plan->threads = T; plan->grid = grid;
    plan->tenor = G;
    plan->smem = smem;
    // the tenor-parallel kernel keeps its path state in shared memory
    plan->state_floats_per_block = G > 0 ? 0 : (size_t)R * nst * ctx->n * T;
    plan->partial_doubles_per_block = (size_t)ctx->n * ctx->ns * 2;
    plan->n_out = ctx->n * ctx->ns * 2;
    plan->stream = ctx->stream;
    plan->device = ctx->device;
    return LLL_OK;
}

}  // namespace lll

extern "C" {

const char *lll_last_error(const lll_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int lll_build_nig_quadrature(lll_nig nig, double xmax, int Q, double *nodes, double *weights)
{
    if (!nodes || !weights || Q < 1) return fail(nullptr, LLL_EINVAL, "null output or Q < 1");
    if (Q > kMaxQP) return fail(nullptr, LLL_EUNSUPPORTED, "Q > 128");
    if (!(nig.alpha > std::fabs(nig.beta)) || !(nig.delta > 0) || !(xmax > 0) || !isfin(xmax))
        return fail(nullptr, LLL_EINVAL, "need alpha > |beta|, delta > 0, xmax > 0");
    if (build_nig_rule(nig.alpha, nig.beta, nig.delta, xmax, Q, nodes, weights) != 0)
        return fail(nullptr, LLL_EINVAL, "quadrature construction failed");
    return LLL_OK;
}

int lll_init(lll_ctx **out, int N, double tenor_delta, const double *L0, int steps_per_period,
             const double *lambda, int driver, lll_nig nig, int Q, const double *nodes,
             const double *weights, void *cuda_stream)
{
    if (!out) return fail(nullptr, LLL_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 2 || N > 4096) return fail(nullptr, LLL_EINVAL, "N must be in [2, 4096]");
    if (!(tenor_delta > 0) || !isfin(tenor_delta)) return fail(nullptr, LLL_EINVAL, "delta <= 0");
    if (steps_per_period < 1 || (long long)(N - 1) * steps_per_period > (1 << 24))
        return fail(nullptr, LLL_EINVAL, "steps_per_period out of range");
    if (!L0 || !lambda) return fail(nullptr, LLL_EINVAL, "L0 or lambda is NULL");
    if (driver != LLL_DRIVER_NIG && driver != LLL_DRIVER_BROWNIAN)
        return fail(nullptr, LLL_EINVAL, "unknown driver");
    const int n = N - 1, S = n * steps_per_period;
    for (int m = 0; m < N; ++m)
        if (!(L0[m] > 0) || !isfin(L0[m])) return fail(nullptr, LLL_EINVAL, "L0 must be finite and > 0");
    for (long long e = 0; e < (long long)S * n; ++e)
        if (!isfin(lambda[e])) return fail(nullptr, LLL_EINVAL, "lambda has NaN/Inf");
    int QP = 0;
    double mu = 0, gam = 0;
    bool domain_warn = false;
    if (driver == LLL_DRIVER_NIG) {
        if (!(nig.alpha > std::fabs(nig.beta)) || !(nig.delta > 0) || !isfin(nig.alpha) ||
            !isfin(nig.beta) || !isfin(nig.delta))
            return fail(nullptr, LLL_EINVAL, "NIG needs alpha > |beta| and delta > 0");
        if (Q < 1 || !nodes || !weights) return fail(nullptr, LLL_EINVAL, "NIG needs Q >= 1 nodes");
        QP = padded_q(Q);
        if (QP < 0) return fail(nullptr, LLL_EUNSUPPORTED, "Q > 128");
        for (int j = 0; j < Q; ++j)
            if (!isfin(nodes[j]) || nodes[j] == 0.0 || !isfin(weights[j]))
                return fail(nullptr, LLL_EINVAL, "nodes must be finite and non-zero");
        gam = std::sqrt(nig.alpha * nig.alpha - nig.beta * nig.beta);
        mu = std::isnan(nig.mu) ? -nig.delta * nig.beta / gam : nig.mu;
        if (!isfin(mu)) return fail(nullptr, LLL_EINVAL, "mu is Inf");
        for (int k = 0; k < S; ++k) {
            double sum = 0;
            for (int l = 0; l < n; ++l) sum += std::fabs(lambda[(size_t)k * n + l]);
            if (sum >= nig.alpha - std::fabs(nig.beta)) domain_warn = true;
        }
    } else {
        Q = 0;
    }

    lll_ctx *c = new lll_ctx();
    c->N = N; c->n = n; c->s = steps_per_period; c->S = S; c->Q = Q; c->QP = QP;
    c->driver = driver; c->delta = tenor_delta; c->h = tenor_delta / steps_per_period;
    c->c = (driver == LLL_DRIVER_BROWNIAN) ? 1.0 : 0.0;
    c->nig = nig; c->mu = mu; c->gam = gam;
    c->stream = (cudaStream_t)cuda_stream;
    c->L0.assign(L0, L0 + N);
    c->lam.assign(lambda, lambda + (size_t)S * n);
    double BN = 1.0;
    for (int m = 0; m < N; ++m) BN /= 1.0 + tenor_delta * L0[m]; // Eq. (i-val) inverted
    c->BN = BN;
    c->chunk_rows = default_chunk_rows(n, QP);

    auto bail = [&](int code) {
        std::string m = c->err;
        free_all(c);
        delete c;
        g_err = m;
        return code;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&c->device)) != cudaSuccess) { cuda_fail(c, e, "cudaGetDevice"); return bail(LLL_ECUDA); }
    if ((e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) {
        cuda_fail(c, e, "cudaDeviceGetAttribute"); return bail(LLL_ECUDA);
    }
    std::vector<float> Z0(n), c0(n);
    std::vector<double> w0(n);
    for (int l = 1; l <= n; ++l) {
        Z0[l - 1] = (float)std::log(L0[l]);
        c0[l - 1] = (float)(std::log(L0[l]) + std::log(tenor_delta));
        w0[l - 1] = tenor_delta * L0[l] / (1.0 + tenor_delta * L0[l]);
    }
    const size_t rows = (size_t)S * n;
    bool ok = dalloc(&c->d_lam, rows) == cudaSuccess && dalloc(&c->d_x, std::max(Q, 1)) == cudaSuccess &&
              dalloc(&c->d_W, std::max(Q, 1)) == cudaSuccess && dalloc(&c->d_w0, n) == cudaSuccess &&
              dalloc(&c->d_b0, rows) == cudaSuccess &&
              dalloc(&c->d_tab, rows * std::max(QP / 4, 1)) == cudaSuccess &&
              dalloc(&c->d_cn, std::max(QP, 4)) == cudaSuccess &&
              dalloc(&c->d_row, rows) == cudaSuccess && dalloc(&c->d_C, rows) == cudaSuccess &&
              dalloc(&c->d_Z0, n) == cudaSuccess &&
              dalloc(&c->d_c0, n) == cudaSuccess;
    if (!ok) { fail(c, LLL_ENOMEM, "cudaMalloc of model tables failed"); return bail(LLL_ENOMEM); }
    for (auto &ev : c->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) { cuda_fail(c, e, "cudaEventCreate"); return bail(LLL_ECUDA); }
    cudaStream_t st = c->stream;
    std::vector<double> xs(std::max(Q, 1), 0.0), ws(std::max(Q, 1), 0.0);
    for (int j = 0; j < Q; ++j) { xs[j] = nodes[j]; ws[j] = weights[j]; }
#define INIT_TRY(expr)                                                                             \
    do {                                                                                           \
        cudaError_t e2 = (expr);                                                                   \
        if (e2 != cudaSuccess) { cuda_fail(c, e2, #expr); return bail(LLL_ECUDA); }               \
    } while (0)
    INIT_TRY(cudaMemcpyAsync(c->d_lam, lambda, sizeof(double) * rows, cudaMemcpyHostToDevice, st));
    INIT_TRY(cudaMemcpyAsync(c->d_x, xs.data(), sizeof(double) * xs.size(), cudaMemcpyHostToDevice, st));
    INIT_TRY(cudaMemcpyAsync(c->d_W, ws.data(), sizeof(double) * ws.size(), cudaMemcpyHostToDevice, st));
    INIT_TRY(cudaMemcpyAsync(c->d_w0, w0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    INIT_TRY(cudaMemcpyAsync(c->d_Z0, Z0.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    INIT_TRY(cudaMemcpyAsync(c->d_c0, c0.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    INIT_TRY(cudaMemsetAsync(c->d_row, 0, sizeof(float4) * rows, st));
    INIT_TRY((cudaError_t)launch_tables(c->d_lam, c->d_x, c->d_W, n, S, Q, QP, c->d_tab, c->d_cn, c->d_row, c->d_C, st));
    INIT_TRY((cudaError_t)launch_frozen_drift(c->d_lam, c->d_x, c->d_W, c->d_w0, n, S, Q, c->c, c->h,
                                              c->d_b0, c->d_row, st));
    // The host vectors above go out of scope: wait for the copies.
    INIT_TRY(cudaStreamSynchronize(st));
#undef INIT_TRY
    *out = c;
    if (domain_warn)
        return fail(c, LLL_EDOMAIN,
                    "sum |lambda| >= alpha - |beta|: the compensator uses the measure truncated to the rule");
    return LLL_OK;
}

int lll_set_product(lll_ctx *ctx, int product)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (product != LLL_PRODUCT_CAPLET && product != LLL_PRODUCT_SWAPTION)
        return fail(ctx, LLL_EINVAL, "unknown product");
    ctx->product = product;
    return LLL_OK;
}

int lll_set_strikes(lll_ctx *ctx, int n_strikes, const double *strikes)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (n_strikes < 1 || n_strikes > 64 || !strikes) return fail(ctx, LLL_EINVAL, "need 1..64 strikes");
    const size_t cnt = (size_t)ctx->n * n_strikes;
    std::vector<float> f(cnt);
    for (size_t e = 0; e < cnt; ++e) {
        if (!isfin(strikes[e])) return fail(ctx, LLL_EINVAL, "strike is NaN/Inf");
        f[e] = (float)strikes[e];
    }
    cudaFree(ctx->d_strikes);
    ctx->d_strikes = nullptr;
    CUDA_TRY(ctx, dalloc(&ctx->d_strikes, cnt));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_strikes, f.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice,
                                  ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->ns = n_strikes;
    ctx->simulated = false;
    return LLL_OK;
}

int lll_set_snapshots(lll_ctx *ctx, uint64_t count, uint64_t stride)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (stride < 1) return fail(ctx, LLL_EINVAL, "stride must be >= 1");
    ctx->snap_stride = stride;
    cudaFree(ctx->d_snap);
    ctx->d_snap = nullptr;
    ctx->n_snap = 0;
    if (count == 0) return LLL_OK;
    const size_t cells = (size_t)ctx->n * ctx->n * count;
    if (count > (1ull << 24)) return fail(ctx, LLL_EINVAL, "snapshot count too large");
    if (dalloc(&ctx->d_snap, cells) != cudaSuccess) return fail(ctx, LLL_ENOMEM, "snapshot buffer");
    ctx->n_snap = count;
    return LLL_OK;
}

int lll_set_launch(lll_ctx *ctx, int threads_per_block, int blocks_per_sm, int chunk_rows,
                   int paths_per_thread, int lanes_per_path)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (threads_per_block != 0 &&
        (threads_per_block < 32 || threads_per_block > kMaxThreads || threads_per_block % 32))
        return fail(ctx, LLL_EINVAL, "threads_per_block must be a multiple of 32 in [32, 256]");
    if (blocks_per_sm < 0 || chunk_rows < 0) return fail(ctx, LLL_EINVAL, "negative launch value");
    if (paths_per_thread < 0 || paths_per_thread > 2)
        return fail(ctx, LLL_EINVAL, "paths_per_thread must be 0 (automatic), 1 or 2");
    if (lanes_per_path != 0 && lanes_per_path != 1 && lanes_per_path != 2 && lanes_per_path != 4)
        return fail(ctx, LLL_EINVAL, "lanes_per_path must be 0 (default), 1, 2 or 4");
    ctx->ppt = paths_per_thread;
    ctx->lpp = lanes_per_path;
    if (threads_per_block) ctx->threads = threads_per_block;
    ctx->blocks_per_sm = blocks_per_sm;
    ctx->chunk_rows = chunk_rows ? std::min(chunk_rows, ctx->n) : default_chunk_rows(ctx->n, ctx->QP);
    return LLL_OK;
}

int lll_set_mapping(lll_ctx *ctx, int mapping, int lanes)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (mapping == LLL_MAP_PATH) {
        ctx->tenor_lanes = 0;
        ctx->step_map = false;
        return LLL_OK;
    }
    if (mapping == LLL_MAP_STEP) {
        ctx->tenor_lanes = 0;
        ctx->step_map = true;
        return LLL_OK;
    }
    if (mapping != LLL_MAP_TENOR) return fail(ctx, LLL_EINVAL, "unknown mapping");
    if (lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
        return fail(ctx, LLL_EINVAL, "lanes must be 4, 8, 16 or 32");
    ctx->tenor_lanes = lanes;
    ctx->step_map = false;
    return LLL_OK;
}

}  // extern "C"

namespace {

// The Picard scheme with its Euler steps in parallel (lll_paths_step.cu):
// chunks of paths through the five kernels, then the fixed-order block sum.
int simulate_step(lll_ctx *ctx, uint64_t first_path, uint64_t paths, uint64_t seed)
{
    LaunchPlan plan;
    int rc = plan_launch(ctx, LLL_PICARD, first_path, paths, seed, &plan, false);
    if (rc != LLL_OK) return rc;
    if (plan.qp == 0 || !step_kernels_supported(plan.qp, ctx->ns))
        return fail(ctx, LLL_EUNSUPPORTED, "the step-parallel mapping needs a node table and at most 64 strikes");
    const int n = ctx->n, S = ctx->S;
    // intermediate arrays of about 4 (S + 2 S n + n^2) bytes per path: chunks within 2 GiB
    const size_t per_path = step_bytes_per_path(n, S);
    uint64_t Pc = std::max<uint64_t>(128, ((size_t(1) << 31) / per_path) / 128 * 128);
    Pc = std::min<uint64_t>(Pc, paths);
    const size_t floats = per_path / 4 * Pc;
    if (floats > ctx->state_cap) {
        cudaFree(ctx->d_state);
        ctx->d_state = nullptr;
        ctx->state_cap = 0;
        if (dalloc(&ctx->d_state, floats) != cudaSuccess) return fail(ctx, LLL_ENOMEM, "step-parallel scratch");
        ctx->state_cap = floats;
    }
    int blocks = 0;
    for (uint64_t c0 = 0; c0 < paths; c0 += Pc) blocks += step_blocks_per_chunk((int)std::min<uint64_t>(Pc, paths - c0));
    const size_t nout = (size_t)plan.n_out;
    if ((size_t)blocks * nout > ctx->partials_cap) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        if (dalloc(&ctx->d_partials, (size_t)blocks * nout) != cudaSuccess) return fail(ctx, LLL_ENOMEM, "partials");
        ctx->partials_cap = (size_t)blocks * nout;
    }
    if (nout > ctx->sums_cap) {
        cudaFree(ctx->d_sums);
        ctx->d_sums = nullptr;
        ctx->sums_cap = 0;
        if (dalloc(&ctx->d_sums, nout) != cudaSuccess) return fail(ctx, LLL_ENOMEM, "sums");
        ctx->sums_cap = nout;
    }
    PathArgs a = plan.args;
    a.snap = ctx->d_snap; a.snap_stride = ctx->snap_stride; a.snap_pitch = ctx->n_snap;
    a.n_snap = ctx->d_snap ? std::min<uint64_t>(ctx->n_snap, (paths + ctx->snap_stride - 1) / ctx->snap_stride) : 0;
    float *dH = ctx->d_state, *Y = dH + (size_t)S * Pc, *Bh = Y + (size_t)S * n * Pc, *Zm = Bh + (size_t)S * n * Pc;
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
    int block0 = 0;
    for (uint64_t c0 = 0; c0 < paths; c0 += Pc) {
        const int pc = (int)std::min<uint64_t>(Pc, paths - c0);
        const cudaError_t e = (cudaError_t)launch_step_chunk(plan.qp, a, c0, pc, dH, Y, Bh, Zm, block0,
                                                             ctx->d_partials, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step-parallel kernels");
        block0 += step_blocks_per_chunk(pc);
    }
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
    const cudaError_t e = (cudaError_t)launch_finalize(ctx->d_partials, blocks, (int)nout, ctx->d_sums, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "finalize launch");
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], ctx->stream));
    ctx->simulated = true;
    ctx->err_pending = false;
    ctx->gemm_err_pending = false;
    ctx->last_paths = paths;
    ctx->last_snap_paths = a.n_snap;
    return LLL_OK;
}

}  // namespace

extern "C" {

int lll_simulate(lll_ctx *ctx, int scheme, uint64_t first_path, uint64_t paths, uint64_t seed)
{
    if (ctx && scheme == LLL_MLP) {
        if (ctx->ns == 0) return fail(ctx, LLL_ESTATE, "lll_set_strikes must come before lll_simulate");
        return simulate_mlp(ctx, first_path, paths, seed);
    }
    if (ctx && (scheme == LLL_EXPAND1 || scheme == LLL_EXPAND2)) {
        if (ctx->ns == 0) return fail(ctx, LLL_ESTATE, "lll_set_strikes must come before lll_simulate");
        if (paths == 0) return fail(ctx, LLL_EINVAL, "paths must be > 0");
        return simulate_expand(ctx, scheme == LLL_EXPAND1 ? 1 : 2, first_path, paths, seed);
    }
    if (ctx && ctx->step_map && (scheme == LLL_PICARD || scheme == LLL_FULL)) {
        if (scheme == LLL_FULL)
            return fail(ctx, LLL_EUNSUPPORTED,
                        "the step-parallel mapping is Picard's: the full scheme's drift reads the simulated rates");
        if (ctx->ns == 0) return fail(ctx, LLL_ESTATE, "lll_set_strikes must come before lll_simulate");
        if (paths == 0) return fail(ctx, LLL_EINVAL, "paths must be > 0");
        return simulate_step(ctx, first_path, paths, seed);
    }
    LaunchPlan plan;
    int rc = plan_launch(ctx, scheme, first_path, paths, seed, &plan);
    if (rc != LLL_OK) return rc;
    const int grid = plan.grid;
    const size_t state_need = plan.state_floats_per_block * grid;
    if (state_need > ctx->state_cap) {
        cudaFree(ctx->d_state);
        ctx->d_state = nullptr;
        ctx->state_cap = 0;
        if (dalloc(&ctx->d_state, state_need) != cudaSuccess) return fail(ctx, LLL_ENOMEM, "state scratch");
        ctx->state_cap = state_need;
    }
    const size_t nout = (size_t)plan.n_out;
    if ((size_t)grid * nout > ctx->partials_cap) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        if (dalloc(&ctx->d_partials, (size_t)grid * nout) != cudaSuccess)
            return fail(ctx, LLL_ENOMEM, "partials");
        ctx->partials_cap = (size_t)grid * nout;
    }
    if (nout > ctx->sums_cap) {
        cudaFree(ctx->d_sums);
        ctx->d_sums = nullptr;
        ctx->sums_cap = 0;
        if (dalloc(&ctx->d_sums, nout) != cudaSuccess) return fail(ctx, LLL_ENOMEM, "sums");
        ctx->sums_cap = nout;
    }
    PathArgs a = plan.args;
    a.partials = ctx->d_partials;
    a.state = ctx->d_state;
    a.snap = ctx->d_snap; a.snap_stride = ctx->snap_stride; a.snap_pitch = ctx->n_snap;
    a.n_snap = ctx->d_snap ? std::min<uint64_t>(ctx->n_snap, (paths + ctx->snap_stride - 1) / ctx->snap_stride) : 0;
    const int QPk = plan.qp, T = plan.threads;
    const size_t smem = plan.smem;
    cudaError_t e;
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
    e = (cudaError_t)launch_plan(plan, a);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "path kernel launch");
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
    e = (cudaError_t)launch_finalize(ctx->d_partials, grid, (int)nout, ctx->d_sums, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "finalize launch");
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], ctx->stream));
    ctx->simulated = true;
    ctx->err_pending = false;
    ctx->gemm_err_pending = false;
    ctx->last_paths = paths;
    ctx->last_snap_paths = a.n_snap;
    return LLL_OK;
}

int lll_get_sums(lll_ctx *ctx, double *sum, double *sumsq, uint64_t *count)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (!ctx->simulated) return fail(ctx, LLL_ESTATE, "no simulation to read");
    if (!sum || !sumsq) return fail(ctx, LLL_EINVAL, "null output");
    const size_t cnt = (size_t)ctx->n * ctx->ns;
    std::vector<double> buf(2 * cnt);
    CUDA_TRY(ctx, cudaMemcpyAsync(buf.data(), ctx->d_sums, sizeof(double) * 2 * cnt,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->gemm_err_pending) {
        int word = 0;
        const cudaError_t e = (cudaError_t)mlp_gemm_take_error(&word, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "GEMM error word");
        ctx->gemm_err_pending = false;
        if (word != 0) {
            ctx->simulated = false;
            return fail(ctx, LLL_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up; results discarded");
        }
    }
    if (ctx->err_pending && ctx->d_err) {
        int word = 0;
        CUDA_TRY(ctx, cudaMemcpy(&word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (word != 0) {
            ctx->simulated = false;
            return fail(ctx, LLL_ETIMEOUT, "a bounded wait of the tensor-core MLP kernel gave up; results discarded");
        }
    }
    for (size_t e = 0; e < cnt; ++e) {
        sum[e] = buf[2 * e];
        sumsq[e] = buf[2 * e + 1];
    }
    if (count) *count = ctx->last_paths;
    return LLL_OK;
}

int lll_price_caplets(lll_ctx *ctx, double *prices, double *stderr_)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (!prices) return fail(ctx, LLL_EINVAL, "prices is NULL");
    const size_t cnt = (size_t)ctx->n * ctx->ns;
    std::vector<double> s1(cnt), s2(cnt);
    uint64_t P = 0;
    int rc = lll_get_sums(ctx, s1.data(), s2.data(), &P);
    if (rc != LLL_OK) return rc;
    const double Pd = (double)P;
    for (size_t e = 0; e < cnt; ++e) {
        const double mean = s1[e] / Pd;
        prices[e] = mean;
        if (stderr_) {
            const double var = std::max(s2[e] / Pd - mean * mean, 0.0) * Pd / std::max(Pd - 1.0, 1.0);
            stderr_[e] = std::sqrt(var / Pd);
        }
    }
    return LLL_OK;
}

int lll_get_paths(lll_ctx *ctx, uint64_t first, uint64_t count, float *out)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (!ctx->simulated || !ctx->d_snap) return fail(ctx, LLL_ESTATE, "no snapshots recorded");
    if (!out) return fail(ctx, LLL_EINVAL, "out is NULL");
    if (first + count > ctx->last_snap_paths) return fail(ctx, LLL_EINVAL, "range beyond recorded snapshots");
    const int n = ctx->n;
    const uint64_t ns = ctx->n_snap; // row pitch of the device buffer
    std::vector<float> buf((size_t)n * n * ns);
    CUDA_TRY(ctx, cudaMemcpyAsync(buf.data(), ctx->d_snap, sizeof(float) * buf.size(),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (uint64_t p = 0; p < count; ++p)
        for (int m = 1; m <= n; ++m)
            for (int l = 1; l <= n; ++l)
                out[((size_t)p * n + (m - 1)) * n + (l - 1)] =
                    (l >= m) ? buf[((size_t)(m - 1) * n + (l - 1)) * ns + first + p] : NAN;
    return LLL_OK;
}

int lll_kernel_ms(lll_ctx *ctx, float *path_kernel_ms, float *simulate_ms)
{
    if (!ctx) return fail(nullptr, LLL_EINVAL, "ctx is NULL");
    if (!ctx->simulated) return fail(ctx, LLL_ESTATE, "no simulation timed");
    CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev[2]));
    float a = 0, b = 0;
    CUDA_TRY(ctx, cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]));
    CUDA_TRY(ctx, cudaEventElapsedTime(&b, ctx->ev[0], ctx->ev[2]));
    if (path_kernel_ms) *path_kernel_ms = a;
    if (simulate_ms) *simulate_ms = b;
    return LLL_OK;
}

void lll_destroy(lll_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
