// lll_mlp_host.cpp -- the learned compensator: network state, training loop
// and the C ABI entry points lll_mlp_*.
//
// All arithmetic runs in the kernels of lll_mlp.cu and lll_mlp_data.cu; this
// file only sizes buffers, orders launches and copies small results.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lll.h"
#include "lll_ctx.h"
#include "lll_internal.h"
#include "lll_mlp.h"

namespace lll {

int mlp_datagen(int QP, const PathArgs &a, const float *Ctab, int R, uint32_t rec_key, float *state,
                float *rec_u, float *rec_y, int *rec_k, cudaStream_t st);
int mlp_gather_vec(const float *rec_u, const float *rec_y, const int *rec_k, uint64_t nrec, int n, int s,
                   double delta, const MlpScales &sc, int in_pad, int O, int rows, uint32_t key0, uint32_t key1,
                   uint32_t step, void *X, float *Y, int *kr, cudaStream_t st);
int mlp_gather(const float *rec_u, const float *rec_y, const int *rec_k, uint64_t nrec, const double *lam,
               int n, int s, double delta, const MlpScales &sc, int in_pad, int rows, uint32_t key0,
               uint32_t key1, uint32_t step, void *X, float *Y, cudaStream_t st);
int mlp_target_moments(const float *rec_y, const int *rec_k, uint64_t nrec, int n, int s, double *part,
                       int blocks, cudaStream_t st);

struct MlpState {
    int hidden = 0, layers = 0, in_dim = 0, in_pad = 0;
    int head = 0;     // 0: one output per (step, rate) row; 1: all rates' outputs per (step) row
    int outputs = 1;  // width of the output layer (head 1: n padded to 16)
    MlpScales sc{};
    size_t n_params = 0;
    std::vector<size_t> offW, offb;
    size_t off_wout = 0, off_bout = 0;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    void *d_ph = nullptr; // BF16 copy of the parameters
    void *d_phT = nullptr; // training: BF16 copies of the weight matrices transposed (same offsets)
    int adam_t = 0;
    bool trained = false;
    // work buffers, sized for `cap` rows
    int cap = 0;
    void *d_X = nullptr;            // bf16 [cap][in_pad]
    float *d_Y = nullptr, *d_out = nullptr, *d_dout = nullptr;
    std::vector<void *> d_H;        // bf16 [cap][hidden], layers
    std::vector<float *> d_Z;       // fp32 [cap][hidden], layers
    float *d_dZ[2] = {nullptr, nullptr};
    void *d_dZh[2] = {nullptr, nullptr};
    float *d_split = nullptr;       // split-K partials
    size_t split_cap = 0;
    double *d_loss = nullptr;       // per-block loss partials
    int loss_cap = 0;
    double *d_acc = nullptr;        // layered scheme: per-block Kahan payoff accumulators
    size_t acc_cap = 0;
    void *d_douth = nullptr;        // head 1: bf16 [cap][outputs] dL/dout
    int *d_kr = nullptr;            // head 1: Euler step of each training row
    double *d_cnt = nullptr;        // head 1: per-block counts of live targets
    float *d_colpart = nullptr;     // column-sum partials [chunks][width + 1]
};

void mlp_free_buffers(MlpState *m)
{
    cudaFree(m->d_X); cudaFree(m->d_Y); cudaFree(m->d_out); cudaFree(m->d_dout);
    cudaFree(m->d_douth); cudaFree(m->d_kr); cudaFree(m->d_cnt);
    m->d_douth = nullptr; m->d_kr = nullptr; m->d_cnt = nullptr;
    for (void *p : m->d_H) cudaFree(p);
    for (float *p : m->d_Z) cudaFree(p);
    m->d_H.clear();
    m->d_Z.clear();
    for (int i = 0; i < 2; ++i) { cudaFree(m->d_dZ[i]); cudaFree(m->d_dZh[i]); m->d_dZ[i] = nullptr; m->d_dZh[i] = nullptr; }
    cudaFree(m->d_split); cudaFree(m->d_loss); cudaFree(m->d_colpart);
    m->d_colpart = nullptr;
    m->d_X = nullptr; m->d_Y = m->d_out = m->d_dout = nullptr; m->d_split = nullptr; m->d_loss = nullptr;
    m->cap = 0; m->split_cap = 0; m->loss_cap = 0;
}

void mlp_free(MlpState *m)
{
    if (!m) return;
    mlp_free_buffers(m);
    cudaFree(m->d_p); cudaFree(m->d_g); cudaFree(m->d_m); cudaFree(m->d_v); cudaFree(m->d_ph); cudaFree(m->d_phT);
    cudaFree(m->d_acc);
    delete m;
}

}  // namespace lll

using namespace lll;

namespace {

int err(lll_ctx *ctx, int code, const std::string &msg) { return record_error(ctx, code, msg.c_str()); }

int cerr(lll_ctx *ctx, cudaError_t e, const char *what)
{
    return err(ctx, LLL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MTRY(expr)                                                                                 \
    do {                                                                                           \
        cudaError_t e_ = (cudaError_t)(expr);                                                      \
        if (e_ != cudaSuccess) return cerr(ctx, e_, #expr);                                        \
    } while (0)

size_t round8(size_t v) { return (v + 7) & ~size_t(7); }

// Flat layout: [W_0 (H x in_pad) | b_0 (H)] [W_l (H x H) | b_l] ... [w_out (H) | b_out]
void layout(MlpState *m)
{
    size_t o = 0;
    m->offW.assign(m->layers, 0);
    m->offb.assign(m->layers, 0);
    for (int l = 0; l < m->layers; ++l) {
        const int din = l == 0 ? m->in_pad : m->hidden;
        m->offW[l] = o;
        o = round8(o + (size_t)m->hidden * din);
        m->offb[l] = o;
        o = round8(o + m->hidden);
    }
    m->off_wout = o;
    o = round8(o + (size_t)m->outputs * m->hidden);
    m->off_bout = o;
    o = round8(o + m->outputs);
    m->n_params = o;
}

int ensure_rows(lll_ctx *ctx, MlpState *m, int rows)
{
    if (rows <= m->cap) return LLL_OK;
    mlp_free_buffers(m);
    const size_t H = m->hidden;
    const size_t O = m->outputs;
    bool ok = cudaMalloc(&m->d_X, 2 * (size_t)rows * m->in_pad) == cudaSuccess &&
              cudaMalloc(&m->d_Y, 4 * (size_t)rows * O) == cudaSuccess &&
              cudaMalloc(&m->d_out, 4 * (size_t)rows * O) == cudaSuccess &&
              cudaMalloc(&m->d_dout, 4 * (size_t)rows * O) == cudaSuccess;
    if (ok && m->head)
        ok = cudaMalloc(&m->d_douth, 2 * (size_t)rows * O) == cudaSuccess &&
             cudaMalloc((void **)&m->d_kr, 4 * (size_t)rows) == cudaSuccess &&
             cudaMalloc((void **)&m->d_cnt, sizeof(double) * (((size_t)rows * O + 127) / 128)) == cudaSuccess;
    for (int l = 0; ok && l < m->layers; ++l) {
        void *hp = nullptr;
        float *zp = nullptr;
        ok = cudaMalloc(&hp, 2 * (size_t)rows * H) == cudaSuccess &&
             cudaMalloc((void **)&zp, 4 * (size_t)rows * H) == cudaSuccess;
        m->d_H.push_back(hp);
        m->d_Z.push_back(zp);
    }
    for (int i = 0; ok && i < 2; ++i)
        ok = cudaMalloc((void **)&m->d_dZ[i], 4 * (size_t)rows * H) == cudaSuccess &&
             cudaMalloc(&m->d_dZh[i], 2 * (size_t)rows * H) == cudaSuccess;
    // loss partials: one per 8 rows (per-rate head), one per 128 outputs (vector head)
    const size_t lb = m->head ? ((size_t)rows * O + 127) / 128 : ((size_t)rows + 7) / 8;
    ok = ok && cudaMalloc((void **)&m->d_loss, sizeof(double) * lb) == cudaSuccess;
    const size_t width = std::max<size_t>(std::max<size_t>(H, O), (size_t)m->in_pad) + 1;
    ok = ok && cudaMalloc((void **)&m->d_colpart, sizeof(float) * width * mlp_colsum_chunks(rows)) == cudaSuccess;
    if (!ok) {
        mlp_free_buffers(m);
        return err(ctx, LLL_ENOMEM, "MLP work buffers");
    }
    m->cap = rows;
    m->loss_cap = lb;
    return LLL_OK;
}

int ensure_split(lll_ctx *ctx, MlpState *m, size_t floats)
{
    if (floats <= m->split_cap) return LLL_OK;
    cudaFree(m->d_split);
    m->d_split = nullptr;
    m->split_cap = 0;
    if (cudaMalloc((void **)&m->d_split, 4 * floats) != cudaSuccess) return err(ctx, LLL_ENOMEM, "split-K buffer");
    m->split_cap = floats;
    return LLL_OK;
}

// Forward pass over `rows` rows already in d_X.  y != nullptr: also residual,
// dL/dout and loss partials.
int forward(lll_ctx *ctx, MlpState *m, int rows, const float *y)
{
    cudaStream_t st = ctx->stream;
    const char *ph = static_cast<const char *>(m->d_ph);
    const void *Hin = m->d_X;
    int din = m->in_pad;
    for (int l = 0; l < m->layers; ++l) {
        // pre-activations are kept only for a backward pass (training: y given)
        MTRY(mlp_gemm(0, 1, 1, Hin, din, ph + 2 * m->offW[l], din, rows, m->hidden, din, 1, nullptr,
                      m->d_p + m->offb[l], nullptr, y ? m->d_Z[l] : nullptr, m->d_H[l], st));
        Hin = m->d_H[l];
        din = m->hidden;
    }
    if (m->head) {
        if (!y && mlp_gemm_kind() == LLL_GEMM_TC) {
            // inference: out^T = W_out H^T + b_out (rates as rows, [outputs][rows]),
            // the layout of the Euler kernel's path state
            MTRY(mlp_gemm(0, 1, 4, ph + 2 * m->off_wout, m->hidden, Hin, m->hidden, m->outputs, rows, m->hidden, 1,
                          m->d_out, m->d_p + m->off_bout, nullptr, nullptr, nullptr, st));
            return LLL_OK;
        }
        // out = H W_out^T (FP32), then bias and, with targets, the masked loss
        MTRY(mlp_gemm(0, 1, 0, Hin, m->hidden, ph + 2 * m->off_wout, m->hidden, rows, m->outputs, m->hidden, 1,
                      m->d_out, nullptr, nullptr, nullptr, nullptr, st));
        MTRY(mlp_vec_loss(m->d_out, m->d_p + m->off_bout, y, m->d_kr, rows, m->outputs, ctx->n, ctx->s, m->d_dout,
                          m->d_douth, y ? m->d_loss : nullptr, m->d_cnt, st));
        return LLL_OK;
    }
    MTRY(mlp_out_loss(Hin, m->hidden, ph + 2 * m->off_wout, m->d_p + m->off_bout, y, rows, m->d_out,
                      m->d_dout, y ? m->d_loss : nullptr, st));
    return LLL_OK;
}

// Backward pass after forward(y): gradients into d_g.
int backward(lll_ctx *ctx, MlpState *m, int rows)
{
    cudaStream_t st = ctx->stream;
    const char *ph = static_cast<const char *>(m->d_ph);
    const char *phT = static_cast<const char *>(m->d_phT);
    const int H = m->hidden, L = m->layers;
    // dW products: K = rows split into ranges of 64 rows (at most 128 CTAs), so
    // that the 128 x din products fill the GPU
    const int splits_req = std::max(1, std::min(128, rows / 64));
    // transposed weights: the dX products then read K-contiguous rows
    const bool tc = mlp_gemm_kind() == LLL_GEMM_TC;
    if (tc) {
        size_t off[6];
        int rr[6], cc[6], cnt = 0;
        for (int l = 1; l < L; ++l) { off[cnt] = m->offW[l]; rr[cnt] = H; cc[cnt] = H; ++cnt; }
        if (m->head) { off[cnt] = m->off_wout; rr[cnt] = m->outputs; cc[cnt] = H; ++cnt; }
        if (cnt > 0) MTRY(mlp_transpose_weights(m->d_ph, m->d_phT, off, rr, cc, cnt, st));
    }
    if (m->head) {
        const int O = m->outputs;
        // dW_out = dout^T H_{L-1} (O x H), db_out = column sums, dZ_{L-1} = (dout W_out) * SiLU'(Z_{L-1})
        const int splits = mlp_splits_used(rows, splits_req);
        int rc = ensure_split(ctx, m, (size_t)splits * O * H);
        if (rc != LLL_OK) return rc;
        MTRY(mlp_gemm(1, 0, 0, m->d_douth, O, m->d_H[L - 1], H, O, H, rows, splits_req, m->d_split, nullptr,
                      nullptr, nullptr, nullptr, st));
        MTRY(mlp_reduce_splits(m->d_split, splits, (size_t)O * H, m->d_g + m->off_wout, st));
        MTRY(mlp_column_sums(m->d_dout, rows, O, m->d_g + m->off_bout, m->d_colpart, st));
        // dZ = (dout W_out) SiLU'(Z): B(k = o, n = h) from the transposed copy [H][O]
        // (tcgen05), or read column-wise from W_out (mma.sync)
        if (tc)
            MTRY(mlp_gemm(0, 1, 2, m->d_douth, O, phT + 2 * m->off_wout, O, rows, H, O, 1, nullptr, nullptr,
                          m->d_Z[L - 1], m->d_dZ[0], m->d_dZh[0], st));
        else
            MTRY(mlp_gemm(0, 0, 2, m->d_douth, O, ph + 2 * m->off_wout, H, rows, H, O, 1, nullptr, nullptr,
                          m->d_Z[L - 1], m->d_dZ[0], m->d_dZh[0], st));
    } else {
        MTRY(mlp_out_weight_grad(m->d_dout, m->d_H[L - 1], rows, H, m->d_g + m->off_wout, m->d_g + m->off_bout,
                                 m->d_colpart, st));
        MTRY(mlp_out_backward(m->d_dout, ph + 2 * m->off_wout, m->d_Z[L - 1], rows, H, m->d_dZ[0], m->d_dZh[0], st));
    }
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
        const int din = l == 0 ? m->in_pad : H;
        const void *Hl = l == 0 ? m->d_X : m->d_H[l - 1];
        const int splits = mlp_splits_used(rows, splits_req);
        int rc = ensure_split(ctx, m, (size_t)splits * H * din);
        if (rc != LLL_OK) return rc;
        // dW_l = dZ_l^T H_l  (M = H, N = din, K = rows)
        MTRY(mlp_gemm(1, 0, 0, m->d_dZh[cur], H, Hl, din, H, din, rows, splits_req, m->d_split, nullptr,
                      nullptr, nullptr, nullptr, st));
        MTRY(mlp_reduce_splits(m->d_split, splits, (size_t)H * din, m->d_g + m->offW[l], st));
        MTRY(mlp_column_sums(m->d_dZ[cur], rows, H, m->d_g + m->offb[l], m->d_colpart, st));
        if (l > 0) {
            // dZ_{l-1} = (dZ_l W_l) * SiLU'(Z_{l-1}), W_l read transposed ([in][out]) by the
            // tcgen05 kernel, column-wise by the mma.sync kernel
            if (tc)
                MTRY(mlp_gemm(0, 1, 2, m->d_dZh[cur], H, phT + 2 * m->offW[l], H, rows, H, H, 1, nullptr, nullptr,
                              m->d_Z[l - 1], m->d_dZ[cur ^ 1], m->d_dZh[cur ^ 1], st));
            else
                MTRY(mlp_gemm(0, 0, 2, m->d_dZh[cur], H, ph + 2 * m->offW[l], H, rows, H, H, 1, nullptr, nullptr,
                              m->d_Z[l - 1], m->d_dZ[cur ^ 1], m->d_dZh[cur ^ 1], st));
            cur ^= 1;
        }
    }
    return LLL_OK;
}

double read_loss(lll_ctx *ctx, MlpState *m, int rows, bool *ok)
{
    if (m->head) {
        // mean over the live targets of the batch (one partial per 128 outputs)
        const size_t lb = ((size_t)rows * m->outputs + 127) / 128;
        std::vector<double> part(lb), cnt(lb);
        *ok = cudaMemcpyAsync(part.data(), m->d_loss, sizeof(double) * lb, cudaMemcpyDeviceToHost, ctx->stream) ==
                  cudaSuccess &&
              cudaMemcpyAsync(cnt.data(), m->d_cnt, sizeof(double) * lb, cudaMemcpyDeviceToHost, ctx->stream) ==
                  cudaSuccess &&
              cudaStreamSynchronize(ctx->stream) == cudaSuccess;
        double s = 0.0, c = 0.0;
        for (int b = 0; b < lb; ++b) { s += part[b]; c += cnt[b]; }
        return c > 0 ? s / c : 0.0;
    }
    const int lb = (rows + 7) / 8;
    std::vector<double> part(lb);
    *ok = cudaMemcpyAsync(part.data(), m->d_loss, sizeof(double) * lb, cudaMemcpyDeviceToHost, ctx->stream) ==
              cudaSuccess &&
          cudaStreamSynchronize(ctx->stream) == cudaSuccess;
    double s = 0.0;
    for (double v : part) s += v;
    return s / rows;
}

float lambda_ref(const lll_ctx *ctx)
{
    double mx = 0.0;
    for (double v : ctx->lam) mx = std::max(mx, std::fabs(v));
    return mx > 0 ? (float)(1.0 / mx) : 1.0f;
}

}  // namespace

extern "C" {

int lll_mlp_init(lll_ctx *ctx, int hidden, int layers, uint64_t seed)
{
    return lll_mlp_init_head(ctx, hidden, layers, 0, seed);
}

int lll_mlp_init_head(lll_ctx *ctx, int hidden, int layers, int head, uint64_t seed)
{
    if (!ctx) return err(nullptr, LLL_EINVAL, "ctx is NULL");
    if (head != 0 && head != 1) return err(ctx, LLL_EINVAL, "head must be 0 (per rate) or 1 (vector)");
    if (ctx->driver != LLL_DRIVER_NIG) return err(ctx, LLL_EINVAL, "the learned compensator needs the NIG driver");
    if ((hidden != 128 && hidden != 256) || layers < 1 || layers > 4)
        return err(ctx, LLL_EINVAL, "hidden must be 128 or 256 and layers 1..4");
    mlp_free(ctx->mlp);
    ctx->mlp = nullptr;
    MlpState *m = new MlpState();
    m->hidden = hidden;
    m->layers = layers;
    m->head = head;
    m->outputs = head ? (ctx->n + 15) / 16 * 16 : 1;
    m->in_dim = head ? 1 + ctx->N : 3 + ctx->N;
    m->in_pad = (int)((m->in_dim + 15) / 16 * 16);
    m->sc.t_scale = (float)(1.0 / (ctx->N * ctx->delta));
    m->sc.i_scale = 1.0f / (float)ctx->n;
    m->sc.lam_scale = lambda_ref(ctx);
    m->sc.u_scale = 4.0f;
    m->sc.y_scale = 1.0f;
    layout(m);
    const size_t P = m->n_params;
    bool ok = cudaMalloc((void **)&m->d_p, 4 * P) == cudaSuccess && cudaMalloc((void **)&m->d_g, 4 * P) == cudaSuccess &&
              cudaMalloc((void **)&m->d_m, 4 * P) == cudaSuccess && cudaMalloc((void **)&m->d_v, 4 * P) == cudaSuccess &&
              cudaMalloc(&m->d_ph, 2 * P) == cudaSuccess && cudaMalloc(&m->d_phT, 2 * P) == cudaSuccess;
    if (!ok) {
        mlp_free(m);
        return err(ctx, LLL_ENOMEM, "MLP parameters");
    }
    // He-uniform initial weights (host RNG, fixed seed), zero biases.
    std::vector<float> hp(P, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l <= layers; ++l) {
        const int din = l == 0 ? m->in_dim : hidden;
        const int rows = l < layers ? hidden : m->outputs;
        const int pitch = l == 0 ? m->in_pad : hidden;
        const size_t off = l < layers ? m->offW[l] : m->off_wout;
        std::uniform_real_distribution<float> U(-std::sqrt(3.0f / din), std::sqrt(3.0f / din));
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < din; ++c) hp[off + (size_t)r * pitch + c] = U(rng);
    }
    ctx->mlp = m;
    cudaStream_t st = ctx->stream;
    MTRY(cudaMemcpyAsync(m->d_p, hp.data(), 4 * P, cudaMemcpyHostToDevice, st));
    MTRY(cudaMemsetAsync(m->d_m, 0, 4 * P, st));
    MTRY(cudaMemsetAsync(m->d_v, 0, 4 * P, st));
    MTRY(cudaMemsetAsync(m->d_g, 0, 4 * P, st));
    MTRY(mlp_to_bf16(m->d_p, P, m->d_ph, st));
    MTRY(cudaStreamSynchronize(st));
    return LLL_OK;
}

int lll_mlp_params(lll_ctx *ctx, int direction, float *params, size_t count, float *scales)
{
    if (!ctx || !ctx->mlp) return err(ctx, LLL_ESTATE, "no network (lll_mlp_init first)");
    MlpState *m = ctx->mlp;
    if (count != m->n_params) return err(ctx, LLL_EINVAL, "parameter count mismatch");
    cudaStream_t st = ctx->stream;
    float sc[5];
    if (direction == 0) {
        if (params) MTRY(cudaMemcpyAsync(params, m->d_p, 4 * count, cudaMemcpyDeviceToHost, st));
        MTRY(cudaStreamSynchronize(st));
        if (scales) {
            sc[0] = m->sc.t_scale; sc[1] = m->sc.i_scale; sc[2] = m->sc.lam_scale; sc[3] = m->sc.u_scale; sc[4] = m->sc.y_scale;
            std::memcpy(scales, sc, sizeof sc);
        }
        return LLL_OK;
    }
    if (params) {
        MTRY(cudaMemcpyAsync(m->d_p, params, 4 * count, cudaMemcpyHostToDevice, st));
        MTRY(mlp_to_bf16(m->d_p, count, m->d_ph, st));
    }
    if (scales) {
        m->sc.t_scale = scales[0]; m->sc.i_scale = scales[1]; m->sc.lam_scale = scales[2];
        m->sc.u_scale = scales[3]; m->sc.y_scale = scales[4];
    }
    MTRY(cudaStreamSynchronize(st));
    m->trained = true;
    return LLL_OK;
}

int lll_mlp_shape(lll_ctx *ctx, int *head, int *outputs)
{
    if (!ctx || !ctx->mlp) return err(ctx, LLL_ESTATE, "no network (lll_mlp_init first)");
    if (head) *head = ctx->mlp->head;
    if (outputs) *outputs = ctx->mlp->outputs;
    return LLL_OK;
}

int lll_mlp_layout(lll_ctx *ctx, size_t *n_params, int *in_dim, int *in_pad, size_t *offsets)
{
    if (!ctx || !ctx->mlp) return err(ctx, LLL_ESTATE, "no network (lll_mlp_init first)");
    MlpState *m = ctx->mlp;
    if (n_params) *n_params = m->n_params;
    if (in_dim) *in_dim = m->in_dim;
    if (in_pad) *in_pad = m->in_pad;
    if (offsets) {
        for (int l = 0; l < m->layers; ++l) { offsets[2 * l] = m->offW[l]; offsets[2 * l + 1] = m->offb[l]; }
        offsets[2 * m->layers] = m->off_wout;
        offsets[2 * m->layers + 1] = m->off_bout;
    }
    return LLL_OK;
}

// Feature rows x[rows][in_dim] (host FP32, converted to BF16) -> out[rows].
// y != NULL: also the MSE loss and, if grads != NULL, its gradient.
int lll_mlp_eval(lll_ctx *ctx, const float *x, const float *y, int rows, float *out, float *grads,
                 double *loss)
{
    if (!ctx || !ctx->mlp) return err(ctx, LLL_ESTATE, "no network (lll_mlp_init first)");
    if (!x || rows < 1) return err(ctx, LLL_EINVAL, "need x and rows >= 1");
    if (grads && !y) return err(ctx, LLL_EINVAL, "gradients need targets");
    MlpState *m = ctx->mlp;
    int rc = ensure_rows(ctx, m, rows);
    if (rc != LLL_OK) return rc;
    cudaStream_t st = ctx->stream;
    std::vector<float> xp((size_t)rows * m->in_pad, 0.0f);
    for (int r = 0; r < rows; ++r)
        std::memcpy(&xp[(size_t)r * m->in_pad], &x[(size_t)r * m->in_dim], 4 * m->in_dim);
    float *tmp = nullptr;
    MTRY(cudaMalloc((void **)&tmp, 4 * xp.size()));
    cudaError_t e = cudaMemcpyAsync(tmp, xp.data(), 4 * xp.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = (cudaError_t)mlp_to_bf16(tmp, xp.size(), m->d_X, st);
    if (e == cudaSuccess && y)
        e = cudaMemcpyAsync(m->d_Y, y, 4 * (size_t)rows * m->outputs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && y && m->head) e = cudaMemsetAsync(m->d_kr, 0, 4 * (size_t)rows, st); // all rates live
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    if (e != cudaSuccess) return cerr(ctx, e, "staging feature rows");
    rc = forward(ctx, m, rows, y ? m->d_Y : nullptr);
    if (rc != LLL_OK) return rc;
    if (grads) {
        rc = backward(ctx, m, rows);
        if (rc != LLL_OK) return rc;
        MTRY(cudaMemcpyAsync(grads, m->d_g, 4 * m->n_params, cudaMemcpyDeviceToHost, st));
    }
    if (out) MTRY(cudaMemcpyAsync(out, m->d_out, 4 * (size_t)rows * m->outputs, cudaMemcpyDeviceToHost, st));
    MTRY(cudaStreamSynchronize(st));
    if (loss && y) {
        bool ok;
        *loss = read_loss(ctx, m, rows, &ok);
        if (!ok) return err(ctx, LLL_ECUDA, "loss readback");
    }
    return LLL_OK;
}

int lll_mlp_train(lll_ctx *ctx, const lll_mlp_cfg *cfg, double *final_loss)
{
    if (!ctx || !cfg) return err(ctx, LLL_EINVAL, "ctx or cfg is NULL");
    if (ctx->driver != LLL_DRIVER_NIG) return err(ctx, LLL_EINVAL, "the learned compensator needs the NIG driver");
    if (cfg->train_paths < 1 || cfg->records_per_path < 1 || cfg->records_per_path > 8 || cfg->epochs < 1 ||
        cfg->batch < 32 || !(cfg->lr > 0))
        return err(ctx, LLL_EINVAL, "bad training configuration");
    int rc;
    if (cfg->head != 0 && cfg->head != 1) return err(ctx, LLL_EINVAL, "head must be 0 or 1");
    if (!ctx->mlp || ctx->mlp->hidden != cfg->hidden || ctx->mlp->layers != cfg->layers ||
        ctx->mlp->head != cfg->head) {
        rc = lll_mlp_init_head(ctx, cfg->hidden, cfg->layers, cfg->head, cfg->seed);
        if (rc != LLL_OK) return rc;
    }
    MlpState *m = ctx->mlp;
    cudaStream_t st = ctx->stream;
    const int n = ctx->n, N = ctx->N, R = cfg->records_per_path;
    const uint64_t P = cfg->train_paths, nrec = P * R;
    // 1. training data from the quadrature full scheme
    LaunchPlan plan;
    rc = plan_launch(ctx, LLL_FULL, 0, P, cfg->seed ^ 0x5EED5EEDull, &plan, false);
    if (rc != LLL_OK) return rc;
    float *state = nullptr, *rec_u = nullptr, *rec_y = nullptr;
    int *rec_k = nullptr;
    double *part = nullptr;
    const int mb = 512;
    bool ok = cudaMalloc((void **)&state, 4 * P * n) == cudaSuccess &&
              cudaMalloc((void **)&rec_u, 4 * nrec * N) == cudaSuccess &&
              cudaMalloc((void **)&rec_y, 4 * nrec * n) == cudaSuccess &&
              cudaMalloc((void **)&rec_k, 4 * nrec) == cudaSuccess &&
              cudaMalloc((void **)&part, sizeof(double) * mb) == cudaSuccess;
    auto cleanup = [&]() { cudaFree(state); cudaFree(rec_u); cudaFree(rec_y); cudaFree(rec_k); cudaFree(part); };
    if (!ok) {
        cleanup();
        return err(ctx, LLL_ENOMEM, "training data buffers");
    }
    cudaError_t e = (cudaError_t)mlp_datagen(ctx->QP, plan.args, ctx->d_C, R, (uint32_t)(cfg->seed * 2654435761u),
                                             state, rec_u, rec_y, rec_k, st);
    std::vector<double> hpart(mb);
    if (e == cudaSuccess) e = (cudaError_t)mlp_target_moments(rec_y, rec_k, nrec, n, ctx->s, part, mb, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hpart.data(), part, sizeof(double) * mb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return cerr(ctx, e, "training data generation");
    }
    double ss = 0.0;
    for (double v : hpart) ss += v;
    // mean number of live rates per record ~ (n+1)/2
    const double pairs = (double)nrec * (n + 1) / 2.0;
    m->sc.y_scale = (float)std::max(std::sqrt(ss / pairs), 1e-30);
    // 2. Adam over batches
    const int B = cfg->batch;
    rc = ensure_rows(ctx, m, B);
    if (rc != LLL_OK) { cleanup(); return rc; }
    // an epoch: every recorded pair (head 0) or every record (head 1) once on average
    const uint64_t steps_per_epoch = std::max<uint64_t>(1, (uint64_t)((m->head ? (double)nrec : pairs) / B));
    const uint64_t total = steps_per_epoch * cfg->epochs;
    const double lr_end = cfg->lr_final > 0 ? cfg->lr_final : cfg->lr;
    double last = 0.0;
    for (uint64_t t = 0; t < total; ++t) {
        const double frac = total > 1 ? (double)t / (total - 1) : 0.0;
        const float lr = (float)(cfg->lr * std::pow(lr_end / cfg->lr, frac));
        if (m->head)
            e = (cudaError_t)mlp_gather_vec(rec_u, rec_y, rec_k, nrec, n, ctx->s, ctx->delta, m->sc, m->in_pad,
                                            m->outputs, B, (uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32),
                                            (uint32_t)t, m->d_X, m->d_Y, m->d_kr, st);
        else
            e = (cudaError_t)mlp_gather(rec_u, rec_y, rec_k, nrec, ctx->d_lam, n, ctx->s, ctx->delta, m->sc,
                                        m->in_pad, B, (uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32),
                                        (uint32_t)t, m->d_X, m->d_Y, st);
        if (e != cudaSuccess) { cleanup(); return cerr(ctx, e, "gather"); }
        rc = forward(ctx, m, B, m->d_Y);
        if (rc == LLL_OK) rc = backward(ctx, m, B);
        if (rc != LLL_OK) { cleanup(); return rc; }
        ++m->adam_t;
        e = (cudaError_t)mlp_adam(m->d_p, m->d_g, m->d_m, m->d_v, m->d_ph, m->n_params, lr, 0.9f, 0.999f,
                                  1e-8f, m->adam_t, st);
        if (e != cudaSuccess) { cleanup(); return cerr(ctx, e, "adam"); }
        if (t + 1 == total) {
            bool okl;
            last = read_loss(ctx, m, B, &okl);
            if (!okl) { cleanup(); return err(ctx, LLL_ECUDA, "loss readback"); }
        }
    }
    e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cerr(ctx, e, "training");
    int word = 0;
    e = (cudaError_t)mlp_gemm_take_error(&word, st);
    if (e != cudaSuccess) return cerr(ctx, e, "GEMM error word");
    if (word) return err(ctx, LLL_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up; training discarded");
    m->trained = true;
    if (final_loss) *final_loss = last;
    return LLL_OK;
}

}  // extern "C"

namespace lll {

// LLL_MLP layer by layer (lll_mlp_layered.cu): any network the training
// kernels run, paths in chunks whose rows (path, live rate) fit the work
// buffers.
int simulate_mlp_layered(lll_ctx *ctx, MlpState *m, uint64_t first_path, uint64_t paths, uint64_t seed)
{
    LaunchPlan plan;
    int rc = plan_launch(ctx, LLL_FULL, first_path, paths, seed, &plan, false);
    if (rc != LLL_OK) return rc;
    const int n = ctx->n, s = ctx->s, S = ctx->S, ns = ctx->ns;
    const int T = mlp_layered_threads();
    // chunk of paths: at most 2^20 rows per step (one per path and live rate,
    // or one per path for the vector head), a multiple of the block size.
    // (Chunks small enough for a layer's activations to stay in L2 measured
    // slower: the products then have too few row tiles per SM.)
    const uint64_t rows_cap = 1u << 20;
    const uint64_t rows_per_path = m->head ? 1 : (uint64_t)n;
    uint64_t Pc = std::max<uint64_t>(T, (rows_cap / rows_per_path) / T * T);
    Pc = std::min<uint64_t>(Pc, (paths + T - 1) / T * T);
    const int grid = (int)(Pc / T);
    rc = ensure_rows(ctx, m, (int)(Pc * rows_per_path));
    if (rc != LLL_OK) return rc;
    const size_t state_need = (size_t)n * Pc;
    if (state_need > ctx->state_cap) {
        cudaFree(ctx->d_state);
        ctx->d_state = nullptr;
        ctx->state_cap = 0;
        if (cudaMalloc((void **)&ctx->d_state, 4 * state_need) != cudaSuccess) return err(ctx, LLL_ENOMEM, "state");
        ctx->state_cap = state_need;
    }
    const size_t cells = (size_t)grid * n * ns;
    if (4 * cells > m->acc_cap) {
        cudaFree(m->d_acc);
        m->d_acc = nullptr;
        m->acc_cap = 0;
        if (cudaMalloc((void **)&m->d_acc, 8 * 4 * cells) != cudaSuccess) return err(ctx, LLL_ENOMEM, "accumulators");
        m->acc_cap = 4 * cells;
    }
    const size_t nout = (size_t)plan.n_out;
    if ((size_t)grid * nout > ctx->partials_cap) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        if (cudaMalloc((void **)&ctx->d_partials, 8 * grid * nout) != cudaSuccess) return err(ctx, LLL_ENOMEM, "partials");
        ctx->partials_cap = (size_t)grid * nout;
    }
    if (nout > ctx->sums_cap) {
        cudaFree(ctx->d_sums);
        ctx->d_sums = nullptr;
        ctx->sums_cap = 0;
        if (cudaMalloc((void **)&ctx->d_sums, 8 * nout) != cudaSuccess) return err(ctx, LLL_ENOMEM, "sums");
        ctx->sums_cap = nout;
    }
    PathArgs a = plan.args;
    a.snap = ctx->d_snap; a.snap_stride = ctx->snap_stride; a.snap_pitch = ctx->n_snap;
    a.n_snap = ctx->d_snap ? std::min<uint64_t>(ctx->n_snap, (paths + ctx->snap_stride - 1) / ctx->snap_stride) : 0;
    cudaStream_t st = ctx->stream;
    MTRY(cudaEventRecord(ctx->ev[0], st));
    MTRY(cudaMemsetAsync(m->d_acc, 0, 8 * 4 * cells, st));
    for (uint64_t c0 = 0; c0 < paths; c0 += Pc) {
        MTRY(cudaMemsetAsync(ctx->d_state, 0, 4 * state_need, st));
        for (int k = 0; k < S; ++k) {
            const int live = n - (k / s + 1) + 1;
            MTRY(launch_mlp_features(a, m->sc, k, (int)Pc, ctx->d_state, m->d_X, m->in_pad, m->head, st));
            rc = forward(ctx, m, (int)(Pc * (m->head ? 1 : live)), nullptr);
            if (rc != LLL_OK) return rc;
            MTRY(launch_mlp_euler(a, ctx->d_C, m->sc.y_scale, k, c0, (int)Pc, ctx->d_state, m->d_out,
                                  m->head ? m->outputs : 0, m->head && mlp_gemm_kind() == LLL_GEMM_TC, m->d_acc,
                                  st));
        }
    }
    MTRY(cudaEventRecord(ctx->ev[1], st));
    MTRY(launch_mlp_acc_to_partials(m->d_acc, cells, ctx->d_partials, st));
    MTRY(launch_finalize(ctx->d_partials, grid, (int)nout, ctx->d_sums, st));
    MTRY(cudaEventRecord(ctx->ev[2], st));
    ctx->simulated = true;
    ctx->err_pending = false;
    ctx->gemm_err_pending = true;
    ctx->last_paths = paths;
    ctx->last_snap_paths = a.n_snap;
    return LLL_OK;
}

// LLL_MLP with a 256-wide vector-head network (lll_mlp_wide.cu): one
// persistent launch, a CTA per SM, 128-path tiles; the CTAs' FP64 Kahan sums
// go to the partials and the fixed-order final reduction.
int simulate_mlp_wide(lll_ctx *ctx, MlpState *m, uint64_t first_path, uint64_t paths, uint64_t seed)
{
    LaunchPlan plan;
    int rc = plan_launch(ctx, LLL_FULL, first_path, paths, seed, &plan, false);
    if (rc != LLL_OK) return rc;
    const uint64_t tiles = (paths + 127) / 128;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)ctx->sm_count));
    const size_t cells = (size_t)grid * ctx->n * ctx->ns;
    if (4 * cells > m->acc_cap) {
        cudaFree(m->d_acc);
        m->d_acc = nullptr;
        m->acc_cap = 0;
        if (cudaMalloc((void **)&m->d_acc, 8 * 4 * cells) != cudaSuccess) return err(ctx, LLL_ENOMEM, "accumulators");
        m->acc_cap = 4 * cells;
    }
    const size_t nout = (size_t)plan.n_out;
    if ((size_t)grid * nout > ctx->partials_cap) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        if (cudaMalloc((void **)&ctx->d_partials, 8 * grid * nout) != cudaSuccess) return err(ctx, LLL_ENOMEM, "partials");
        ctx->partials_cap = (size_t)grid * nout;
    }
    if (nout > ctx->sums_cap) {
        cudaFree(ctx->d_sums);
        ctx->d_sums = nullptr;
        ctx->sums_cap = 0;
        if (cudaMalloc((void **)&ctx->d_sums, 8 * nout) != cudaSuccess) return err(ctx, LLL_ENOMEM, "sums");
        ctx->sums_cap = nout;
    }
    if (!ctx->d_err && cudaMalloc((void **)&ctx->d_err, sizeof(int)) != cudaSuccess)
        return err(ctx, LLL_ENOMEM, "error word");
    PathArgs a = plan.args;
    a.partials = ctx->d_partials;
    a.snap = ctx->d_snap; a.snap_stride = ctx->snap_stride; a.snap_pitch = ctx->n_snap;
    a.n_snap = ctx->d_snap ? std::min<uint64_t>(ctx->n_snap, (paths + ctx->snap_stride - 1) / ctx->snap_stride) : 0;
    MlpArgs g{};
    g.wh = static_cast<const __nv_bfloat16 *>(m->d_ph);
    g.wp = m->d_p;
    for (int l = 0; l < m->layers; ++l) { g.offW[l] = m->offW[l]; g.offb[l] = m->offb[l]; }
    g.off_wout = m->off_wout;
    g.off_bout = m->off_bout;
    g.sc = m->sc;
    g.Ctab = ctx->d_C;
    g.in_pad = m->in_pad;
    g.err = ctx->d_err;
    g.stall_mma = ctx->inject == LLL_INJECT_MMA_STALL ? 1 : 0;
    ctx->inject = LLL_INJECT_NONE; // one launch only
    cudaStream_t st = ctx->stream;
    MTRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
    MTRY(cudaMemsetAsync(m->d_acc, 0, 8 * 4 * cells, st));
    MTRY(cudaEventRecord(ctx->ev[0], st));
    MTRY(launch_mlp_wide(m->layers, m->in_pad, m->outputs, grid, st, a, g, m->d_acc));
    MTRY(cudaEventRecord(ctx->ev[1], st));
    MTRY(launch_mlp_acc_to_partials(m->d_acc, cells, ctx->d_partials, st));
    MTRY(launch_finalize(ctx->d_partials, grid, (int)nout, ctx->d_sums, st));
    MTRY(cudaEventRecord(ctx->ev[2], st));
    ctx->simulated = true;
    ctx->err_pending = true;
    ctx->gemm_err_pending = false;
    ctx->last_paths = paths;
    ctx->last_snap_paths = a.n_snap;
    return LLL_OK;
}

// lll_simulate(LLL_MLP): the full scheme with the network's compensator.
int simulate_mlp(lll_ctx *ctx, uint64_t first_path, uint64_t paths, uint64_t seed)
{
    MlpState *m = ctx->mlp;
    if (!m || !m->trained) return err(ctx, LLL_ESTATE, "LLL_MLP needs lll_mlp_train or lll_mlp_load first");
    bool vec_tc = false;
    if (m->head) {
        vec_tc = mlp_tc_vec_supported(m->hidden, m->layers, m->in_pad, m->outputs, ctx->n) &&
                 mlp_tc_vec_smem(m->layers, m->in_pad, ctx->n, ctx->ns) <= 227 * 1024;
        const bool wide = mlp_wide_supported(m->hidden, m->layers, m->in_pad, m->outputs, ctx->n, ctx->ns, ctx->product);
        if (ctx->mlp_kernel == LLL_MLP_KERNEL_WARP)
            return err(ctx, LLL_EUNSUPPORTED, "the mma.sync kernel has no vector head");
        if (ctx->mlp_kernel == LLL_MLP_KERNEL_TC && !vec_tc && !wide)
            return err(ctx, LLL_EUNSUPPORTED, "the tcgen05 vector-head kernels do not support this network");
        if (ctx->mlp_kernel == LLL_MLP_KERNEL_LAYERED || (!vec_tc && !wide))
            return simulate_mlp_layered(ctx, m, first_path, paths, seed);
        if (!vec_tc) return simulate_mlp_wide(ctx, m, first_path, paths, seed);
    }
    const size_t smem_tc = vec_tc ? mlp_tc_vec_smem(m->layers, m->in_pad, ctx->n, ctx->ns)
                                  : mlp_tc_smem(m->layers, m->in_pad, ctx->n, ctx->ns);
    const bool tc_ok = vec_tc || (mlp_tc_supported(m->hidden, m->layers, m->in_pad) && smem_tc <= 227 * 1024);
    const bool warp_ok = mlp_path_supported(m->hidden, m->layers, m->in_pad) &&
                         mlp_path_smem(m->layers, m->in_pad, ctx->n, ctx->ns) <= 227 * 1024;
    bool use_tc;
    if (ctx->mlp_kernel == LLL_MLP_KERNEL_TC) {
        if (!tc_ok) return err(ctx, LLL_EUNSUPPORTED, "the tcgen05 MLP kernel does not support this network");
        use_tc = true;
    } else if (ctx->mlp_kernel == LLL_MLP_KERNEL_WARP) {
        if (!warp_ok) return err(ctx, LLL_EUNSUPPORTED, "the mma.sync MLP kernel handles hidden = 128 and N <= 61");
        use_tc = false;
    } else if (ctx->mlp_kernel == LLL_MLP_KERNEL_LAYERED || (!tc_ok && !warp_ok)) {
        return simulate_mlp_layered(ctx, m, first_path, paths, seed);
    } else {
        use_tc = tc_ok;
    }
    LaunchPlan plan;
    int rc = plan_launch(ctx, LLL_FULL, first_path, paths, seed, &plan, false);
    if (rc != LLL_OK) return rc;
    const size_t smem = use_tc ? smem_tc : mlp_path_smem(m->layers, m->in_pad, ctx->n, ctx->ns);
    int occ = 0;
    if (vec_tc) MTRY(mlp_tc_vec_occupancy(m->layers, m->in_pad, smem, &occ));
    else if (use_tc) MTRY(mlp_tc_occupancy(m->layers, m->in_pad, smem, &occ));
    else MTRY(mlp_path_occupancy(m->layers, m->in_pad, smem, &occ));
    if (occ < 1) return err(ctx, LLL_EUNSUPPORTED, "MLP kernel does not fit on an SM");
    if (use_tc && !ctx->d_err) {
        if (cudaMalloc((void **)&ctx->d_err, sizeof(int)) != cudaSuccess) return err(ctx, LLL_ENOMEM, "error word");
    }
    const int T = use_tc ? mlp_tc_paths_per_block() : mlp_path_threads();
    const uint64_t tiles = (paths + T - 1) / T;
    const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)occ * ctx->sm_count);
    const size_t state_need = (size_t)grid * ctx->n * T;
    if (state_need > ctx->state_cap) {
        cudaFree(ctx->d_state);
        ctx->d_state = nullptr;
        ctx->state_cap = 0;
        if (cudaMalloc((void **)&ctx->d_state, 4 * state_need) != cudaSuccess) return err(ctx, LLL_ENOMEM, "state");
        ctx->state_cap = state_need;
    }
    const size_t nout = (size_t)plan.n_out;
    if ((size_t)grid * nout > ctx->partials_cap) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partials_cap = 0;
        if (cudaMalloc((void **)&ctx->d_partials, 8 * grid * nout) != cudaSuccess) return err(ctx, LLL_ENOMEM, "partials");
        ctx->partials_cap = (size_t)grid * nout;
    }
    if (nout > ctx->sums_cap) {
        cudaFree(ctx->d_sums);
        ctx->d_sums = nullptr;
        ctx->sums_cap = 0;
        if (cudaMalloc((void **)&ctx->d_sums, 8 * nout) != cudaSuccess) return err(ctx, LLL_ENOMEM, "sums");
        ctx->sums_cap = nout;
    }
    PathArgs a = plan.args;
    a.state = ctx->d_state;
    a.partials = ctx->d_partials;
    a.snap = ctx->d_snap; a.snap_stride = ctx->snap_stride; a.snap_pitch = ctx->n_snap;
    a.n_snap = ctx->d_snap ? std::min<uint64_t>(ctx->n_snap, (paths + ctx->snap_stride - 1) / ctx->snap_stride) : 0;
    MlpArgs g{};
    g.wh = static_cast<const __nv_bfloat16 *>(m->d_ph);
    g.wp = m->d_p;
    for (int l = 0; l < m->layers; ++l) { g.offW[l] = m->offW[l]; g.offb[l] = m->offb[l]; }
    g.off_wout = m->off_wout;
    g.off_bout = m->off_bout;
    g.sc = m->sc;
    g.Ctab = ctx->d_C;
    g.in_pad = m->in_pad;
    g.err = ctx->d_err;
    g.stall_mma = (use_tc && ctx->inject == LLL_INJECT_MMA_STALL) ? 1 : 0;
    if (use_tc) ctx->inject = LLL_INJECT_NONE; // one launch only
    if (use_tc) {
        MTRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
        ctx->err_pending = true;
        ctx->gemm_err_pending = false;
    }
    MTRY(cudaEventRecord(ctx->ev[0], ctx->stream));
    if (vec_tc) MTRY(launch_mlp_tc_vec(m->layers, m->in_pad, grid, smem, ctx->stream, a, g));
    else if (use_tc) MTRY(launch_mlp_tc(m->layers, m->in_pad, grid, smem, ctx->stream, a, g));
    else MTRY(launch_mlp_path(m->layers, m->in_pad, grid, smem, ctx->stream, a, g));
    MTRY(cudaEventRecord(ctx->ev[1], ctx->stream));
    MTRY(launch_finalize(ctx->d_partials, grid, (int)nout, ctx->d_sums, ctx->stream));
    MTRY(cudaEventRecord(ctx->ev[2], ctx->stream));
    ctx->simulated = true;
    ctx->last_paths = paths;
    ctx->last_snap_paths = a.n_snap;
    return LLL_OK;
}

}  // namespace lll

extern "C" {

int lll_mlp_set_kernel(lll_ctx *ctx, int kind)
{
    if (!ctx) return err(nullptr, LLL_EINVAL, "ctx is NULL");
    if (kind != LLL_MLP_KERNEL_AUTO && kind != LLL_MLP_KERNEL_WARP && kind != LLL_MLP_KERNEL_TC &&
        kind != LLL_MLP_KERNEL_LAYERED)
        return err(ctx, LLL_EINVAL, "unknown MLP kernel");
    ctx->mlp_kernel = kind;
    return LLL_OK;
}

int lll_inject(lll_ctx *ctx, int what)
{
    if (!ctx) return err(nullptr, LLL_EINVAL, "ctx is NULL");
    if (what != LLL_INJECT_NONE && what != LLL_INJECT_MMA_STALL) return err(ctx, LLL_EINVAL, "unknown injection");
    ctx->inject = what;
    return LLL_OK;
}

int lll_mlp_save(lll_ctx *ctx, const char *path)
{
    if (!ctx || !ctx->mlp || !path) return err(ctx, LLL_EINVAL, "no network or path");
    MlpState *m = ctx->mlp;
    std::vector<float> p(m->n_params);
    float sc[5];
    int rc = lll_mlp_params(ctx, 0, p.data(), p.size(), sc);
    if (rc != LLL_OK) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return err(ctx, LLL_EINVAL, std::string("cannot open ") + path);
    const char magic[8] = {'L', 'L', 'L', 'M', 'L', 'P', '0', '1'};
    const int32_t hdr[4] = {m->hidden, m->layers, m->in_dim, ctx->N};
    const uint64_t cnt = p.size();
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 4, f) == 4 && std::fwrite(sc, 4, 5, f) == 5 &&
              std::fwrite(&cnt, 8, 1, f) == 1 && std::fwrite(p.data(), 4, cnt, f) == cnt;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LLL_OK : err(ctx, LLL_EINVAL, "write failed");
}

int lll_mlp_load(lll_ctx *ctx, const char *path)
{
    if (!ctx || !path) return err(ctx, LLL_EINVAL, "ctx or path is NULL");
    FILE *f = std::fopen(path, "rb");
    if (!f) return err(ctx, LLL_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    float sc[5];
    uint64_t cnt = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "LLLMLP01", 8) == 0 &&
              std::fread(hdr, 4, 4, f) == 4 && std::fread(sc, 4, 5, f) == 5 && std::fread(&cnt, 8, 1, f) == 1;
    std::vector<float> p;
    if (ok && cnt < (1ull << 28)) {
        p.resize(cnt);
        ok = std::fread(p.data(), 4, cnt, f) == cnt;
    } else {
        ok = false;
    }
    std::fclose(f);
    if (!ok) return err(ctx, LLL_EINVAL, "not a network file");
    if (hdr[3] != ctx->N) return err(ctx, LLL_EINVAL, "network was trained for another tenor count");
    if (hdr[2] != 3 + ctx->N && hdr[2] != 1 + ctx->N) return err(ctx, LLL_EINVAL, "unknown input width");
    int rc = lll_mlp_init_head(ctx, hdr[0], hdr[1], hdr[2] == 1 + ctx->N ? 1 : 0, 0);
    if (rc != LLL_OK) return rc;
    return lll_mlp_params(ctx, 1, p.data(), p.size(), sc);
}

}  // extern "C"
