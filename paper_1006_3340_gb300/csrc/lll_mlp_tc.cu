// lll_mlp_tc.cu -- the full scheme with the learned compensator (LLL_MLP) on
// the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Same method as lll_mlp_path.cu: Euler steps of Eq. (log-LIB-SDE-2) with the
// drift of Eq. (LIBOR-drift-PT), the jump compensator of every live rate being
// A_i = C_i + s_y f(x_i) with the feature row
// x_i = (t s_t, i s_i, lambda_i s_lam, u_0 .. u_{N-1}) of the log-rates at t_k
// and f the trained network (SiLU hidden layers, BF16 weights and
// activations, FP32 accumulation).
//
// Roles of a CTA (544 threads), per-rate network (mlp_tc_kernel):
//  * warp 16: allocates 512 TMEM columns and, from one lane, issues the
//    products of both path tiles in turn (128 paths each, one per TMEM lane).
//    Per live rate and tile: the first layer from the feature rows in shared
//    memory (128-byte swizzled, K-major), then the hidden layers with the
//    previous layer's BF16 activations as the A operand in TMEM; every product
//    accumulates FP32 into the tile's 128-column accumulator.  t, i and
//    lambda_i are the same for every path of a (step, rate), so they enter the
//    first layer as a per-rate bias and the feature rows change once per step.
//  * warps 0-15: epilogue, warp 4 cq + q: TMEM lane quadrant q and column
//    quarter cq.  Every warp works on both tiles, one layer at a time in turn:
//    it reads 32 accumulator columns, adds the bias, applies SiLU and writes
//    the next layer's activations with tcgen05.st, or forms its quarter of the
//    output dot product.  The cq = 0 thread of a row owns the row's path in
//    both tiles: increments, feature rows, the Euler step (one rate late, off
//    the products' critical path) and the caplet bookkeeping.  Path state and
//    the step's lambda and C rows are kept in shared memory.
// Weights stay in shared memory for the whole launch.  Hand-offs use
// mbarriers (operand ready: one arrival per epilogue warp; accumulator ready:
// tcgen05.commit; output partials ready).  Every wait first tests the phase
// and then waits boundedly: on timeout the CTA sets an error word, abandons
// its work and releases its tensor memory.  The vector-head kernel
// (mlp_tc_vec_kernel) below shares this layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lll_device.cuh"
#include "lll_internal.h"
#include "lll_mlp.h"
#include "lll_tc.cuh"

namespace lll {
namespace {

constexpr int kH = 128;               // hidden width
constexpr int kRows = 128;            // rows (paths) per warpgroup tile
constexpr int kGroups = 2;            // path tiles in flight per CTA
constexpr int kEpiWarps = 8 * kGroups; // 4 TMEM lane quadrants x 4 column quarters (vector head: x 2 halves x 2 tiles)
constexpr int kThreads = (kEpiWarps + 1) * 32;
constexpr int kTileBytes = kRows * 128; // one 64-wide K block of a 128-row operand
using namespace tc;

// Instruction descriptor of the hidden layers: D FP32, A and B BF16, both K-major, M = 128, N = kH.
constexpr uint32_t kIdesc = idesc_m128(kH);
__host__ __device__ constexpr uint32_t idesc_n(int n) { return idesc_m128(n); }

// Byte offset of the 16-byte chunk c8 (0..7) of K block kb in row r of a 128-row operand.
__device__ __forceinline__ uint32_t chunk_off(int r, int kb, int c8) { return (uint32_t)(kb * kTileBytes) + swz(r, c8); }

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t acc) { mma_ss(d, ad, bd, kIdesc, acc); }
__device__ __forceinline__ void mma_bf16_ts(uint32_t d, uint32_t at, uint64_t bd, uint32_t acc) { mma_ts(d, at, bd, kIdesc, acc); }

// Bias + SiLU of 8 accumulator values: with z = v + b and hz = z / 2 (from
// the half bias hb), SiLU(z) = z sigma(z) = hz + hz tanh(hz), the same
// function as the training kernels' z (1 + tanh(z / 2)) / 2 (one MUFU
// operation and two f32x2 FMAs per pair).  hb is 16-byte aligned: the eight
// biases come in two 128-bit shared loads (one wavefront each, all lanes
// reading the same address).
__device__ __forceinline__ void silu8(const uint32_t *v, const float *hb, float (&sv)[8])
{
    const float4 b0 = *reinterpret_cast<const float4 *>(hb), b1 = *reinterpret_cast<const float4 *>(hb + 4);
    const float hbv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        const float2 hz = __ffma2_rn(make_float2(__uint_as_float(v[e]), __uint_as_float(v[e + 1])),
                                     make_float2(0.5f, 0.5f), make_float2(hbv[e], hbv[e + 1]));
        const float2 t = make_float2(tanh_approx(hz.x), tanh_approx(hz.y));
        const float2 r = __ffma2_rn(hz, t, hz);
        sv[e] = r.x;
        sv[e + 1] = r.y;
    }
}

// Shared-memory plan; operand tiles first (1024-byte aligned).
struct TcLayout {
    uint32_t w0, w, u, bias, w0c, hbw, wout, bars, misc, opart, red, bsum, state, lc, total;
};

__host__ __device__ inline TcLayout tc_layout(int L, int KB0, int n, int ns)
{
    TcLayout t;
    uint32_t o = 0;
    t.w0 = o; o += KB0 * kTileBytes;             // W_0: H rows x 64 KB0 columns
    t.w = o; o += (L - 1) * 2 * kTileBytes;       // W_1 .. W_{L-1}: H rows x 128 columns
    t.u = o; o += kGroups * KB0 * kTileBytes;     // feature rows, per tile (hidden activations live in TMEM)
    t.bias = o; o += L * kH * 4;                  // b_0 / 2 .. b_{L-1} / 2
    t.w0c = o; o += 3 * kH * 4;                   // W_0 columns of t, i, lambda, halved
    t.hbw = o; o += kEpiWarps * 64 * 4;           // per warp: first-layer half biases of two rates
    t.wout = o; o += kH * 4;                      // output weights (BF16 values)
    t.bars = o; o += 12 * 8;                      // mbarriers
    t.misc = o; o += 16;                          // TMEM base, abort word
    t.opart = o; o += kGroups * 3 * kRows * 4;    // output partials of column quarters 1..3, per tile
    o = (o + 15) & ~15u;
    t.red = o; o += 2 * 4 * ns * 2 * 8;           // 4 owner warps' payoff sums, two buffers
    t.bsum = o; o += n * ns * 4 * 8;              // Kahan accumulators
    t.state = o; o += n * kGroups * kRows * 4;    // log-rate offsets of the CTA's paths, [rate][path]
    t.lc = o; o += kEpiWarps * 2 * ((n + 31) & ~31) * 4; // per warp: lambda_i(t_k) and C_i(t_k) of the step
    t.total = o + 1024;                           // slack for aligning the base
    return t;
}

template <int L, int KB0>
__global__ void __launch_bounds__(kThreads, 1) mlp_tc_kernel(const PathArgs a, const MlpArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    const int n = a.n, s = a.s, S = a.S, ns = a.ns;
    const TcLayout lay = tc_layout(L, KB0, n, ns);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = saddr(sm);
    float *bias = reinterpret_cast<float *>(sm + lay.bias);
    float *wout = reinterpret_cast<float *>(sm + lay.wout);
    float *w0c = reinterpret_cast<float *>(sm + lay.w0c);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + lay.bars);
    // Operand-ready barriers, one arrival per epilogue warp: feature rows and a
    // free accumulator (first layer) and activations (hidden layers) have
    // separate barriers, so a warp never arrives twice on one barrier before
    // its phase completed (every arrival on either is preceded by a wait for
    // the previous product).
    uint64_t *opu = bars + 0;  // [kGroups] feature rows written, accumulator free
    uint64_t *opx = bars + 2;  // [kGroups] activations ready
    uint64_t *dnb = bars + 4;  // [kGroups] accumulator ready (commit)
    uint64_t *outb = bars + 6; // [kGroups] output partials of column quarters 1..3 written (12 arrivals)
    uint64_t *payb = bars + 8; // payoff partials written (the 4 path-owning warps; payb[0] only)
    uint64_t *finb = bars + 10; // all MMAs complete (commit)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + lay.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + lay.misc + 4);
    float *opart = reinterpret_cast<float *>(sm + lay.opart);
    double *red = reinterpret_cast<double *>(sm + lay.red);
    double *bsum = reinterpret_cast<double *>(sm + lay.bsum);
    const int in_pad = KB0 * 64 >= g.in_pad ? g.in_pad : KB0 * 64;

    // ---- stage the weights into the swizzled operand layout ----
    for (int l = 0; l < L; ++l) {
        const int din = l == 0 ? in_pad : kH;
        const int chunks = l == 0 ? KB0 * 8 : 16; // 16-byte chunks per row
        const __nv_bfloat16 *W = g.wh + g.offW[l];
        const uint32_t base = l == 0 ? lay.w0 : lay.w + (l - 1) * 2 * kTileBytes;
        for (int e = tid; e < kH * chunks; e += kThreads) {
            const int h = e / chunks, c = e % chunks;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (c * 8 < din) v = *reinterpret_cast<const uint4 *>(W + (size_t)h * din + c * 8);
            if (l == 0 && c == 0) {
                // columns t, i, lambda_i: the same for every path of a (step, rate),
                // so they enter through the per-rate bias instead of the product
                v.x = 0u;
                v.y &= 0xffff0000u;
            }
            *reinterpret_cast<uint4 *>(sm + base + chunk_off(h, c >> 3, c & 7)) = v;
        }
    }
    for (int e = tid; e < L * kH; e += kThreads) bias[e] = 0.5f * g.wp[g.offb[e / kH] + e % kH]; // half biases
    for (int e = tid; e < kH; e += kThreads) wout[e] = __bfloat162float(g.wh[g.off_wout + e]);
    for (int e = tid; e < 3 * kH; e += kThreads)
        w0c[e] = 0.5f * __bfloat162float(g.wh[g.offW[0] + (size_t)(e % kH) * g.in_pad + e / kH]);
    for (int e = tid; e < 4 * n * ns; e += kThreads) bsum[e] = 0.0;
    if (tid == 0) {
        for (int gi = 0; gi < kGroups; ++gi) {
            mbar_init(&opu[gi], kEpiWarps); // every epilogue warp
            mbar_init(&opx[gi], kEpiWarps);
            mbar_init(&dnb[gi], 1);
            mbar_init(&outb[gi], 12);       // the warps of column quarters 1..3
            mbar_init(&payb[gi], 4);        // the 4 path-owning warps (payb[0] only)
        }
        mbar_init(finb, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(kGroups * 2 * kH));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;
    const uint64_t ntiles = (a.paths + kGroups * kRows - 1) / (kGroups * kRows);

    if (warp == kEpiWarps) {
        // ---------------- MMA issuer ----------------
        // Per live rate and tile: the first layer (feature rows in shared
        // memory; the rate's own inputs t, i, lambda_i enter through a per-rate
        // bias, so the rows change once per step), then the hidden layers with
        // the activations as the A operand in tensor memory.  Each tile's
        // accumulator is TMEM columns [128 gi, 128 gi + 128), its activations
        // [256 + 64 gi, 256 + 64 gi + 64).  The tiles are served in turn.
        if (lane == 0) {
            uint32_t phu[kGroups] = {0, 0}, phx[kGroups] = {0, 0};
            bool ok = !g.stall_mma; // stalled: nothing is issued, the epilogue's waits run out
            auto issue = [&](int gi, int l) {
                uint64_t *ob = l == 0 ? &opu[gi] : &opx[gi];
                uint32_t &ph = l == 0 ? phu[gi] : phx[gi];
                if (!mbar_wait(ob, ph, abort, g.err)) return false;
                ph ^= 1;
                tc_after();
                const uint32_t d = tmem + gi * kH;
                const uint32_t bbase = sbase + (l == 0 ? lay.w0 : lay.w + (l - 1) * 2 * kTileBytes);
                if (l == 0) {
                    const uint32_t abase = sbase + lay.u + gi * KB0 * kTileBytes;
                    for (int ks = 0; ks < in_pad / 16; ++ks) {
                        const uint32_t off = (ks >> 2) * kTileBytes + (ks & 3) * 32;
                        mma_bf16(d, sdesc(abase + off), sdesc(bbase + off), ks > 0);
                    }
                } else {
                    const uint32_t at = tmem + 2 * kH + gi * (kH / 2);
                    for (int ks = 0; ks < kH / 16; ++ks) {
                        const uint32_t off = (ks >> 2) * kTileBytes + (ks & 3) * 32;
                        mma_bf16_ts(d, at + ks * 8, sdesc(bbase + off), ks > 0);
                    }
                }
                mma_commit(&dnb[gi]);
                return true;
            };
            for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x)
                for (int k = 0; ok && k < S; ++k) {
                    const int live = n - (k / s + 1) + 1;
                    for (int r = 0; ok && r < live; ++r)
                        for (int l = 0; ok && l < L; ++l)
                            for (int gi = 0; ok && gi < kGroups; ++gi) ok = issue(gi, l);
                }
            // drain: the commit below completes only after every MMA issued above
            mma_commit(finb);
            volatile int dummy_abort = 0;
            mbar_wait(finb, 0, &dummy_abort, g.err);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps ----------------
        // warp = 4 cq + q4: TMEM lane quadrant q4 (row 32 q4 + lane of each tile)
        // and column quarter cq (columns 32 cq .. 32 cq + 31).  Every warp works
        // on both tiles, one layer at a time in tile order, so that one tile's
        // product runs on the tensor pipe while the other tile's epilogue runs.
        // The cq = 0 thread of a row owns that row's path in both tiles.
        const int cq = warp >> 2, q4 = warp & 3;
        const int row = q4 * 32 + lane;          // TMEM lane = tile row
        const int T = kGroups * kRows;           // paths per CTA tile pair
        const bool owner = cq == 0;
        const uint32_t dq = tmem + ((uint32_t)(q4 * 32) << 16) + cq * 32;          // + tile * kH: accumulator
        const uint32_t aq = tmem + ((uint32_t)(q4 * 32) << 16) + 2 * kH + cq * 16; // + tile * kH / 2: activations
        float *hbw = reinterpret_cast<float *>(sm + lay.hbw) + warp * 64; // two rate slots of 32
        float *st = reinterpret_cast<float *>(sm + lay.state) + row; // [rate][path]: + (i - 1) T + tile * kRows
        const int npad = (n + 31) & ~31;
        float *lw = reinterpret_cast<float *>(sm + lay.lc) + (size_t)warp * 2 * npad; // lambda_i, then C_i
        const float h = a.h;
        const float b_out = g.wp[g.off_bout];
        uint32_t phd[kGroups] = {0, 0}, pho[kGroups] = {0, 0}, php = 0;
        int mcount = 0;
        bool ok = true;
        for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            uint64_t p[kGroups], sidx[kGroups];
            bool active[kGroups];
#pragma unroll
            for (int gi = 0; gi < kGroups; ++gi) {
                const uint64_t lp = tile * (uint64_t)T + gi * kRows + row;
                active[gi] = lp < a.paths;
                p[gi] = a.first_path + lp;
                sidx[gi] = ~0ull;
                if (owner && a.snap != nullptr && active[gi] && lp % a.snap_stride == 0 &&
                    lp / a.snap_stride < a.n_snap)
                    sidx[gi] = lp / a.snap_stride;
                if (owner)
                    for (int l = 0; l < n; ++l) st[(size_t)l * T + gi * kRows] = 0.0f;
            }

            for (int k = 0; ok && k < S; ++k) {
                const int imin = k / s + 1;
                const bool mat = (k + 1) % s == 0;
                float dH[kGroups] = {0.0f, 0.0f};
                const float xt = (float)k * h * g.sc.t_scale;
                if (owner) {
#pragma unroll
                    for (int gi = 0; gi < kGroups; ++gi) {
                        const float *sg = st + gi * kRows;
                        unsigned char *ug = sm + lay.u + gi * KB0 * kTileBytes;
                        dH[gi] = draw_increment(a, p[gi], (uint32_t)k);
                        // feature row of this path at t_k: u_m at column 3 + m (u_0 = 0); the
                        // columns of t, i, lambda_i stay zero (they enter through the per-rate bias)
                        for (int c8 = 0; c8 < KB0 * 8; ++c8) {
                            float f[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int m = c8 * 8 + e - 3;
                                f[e] = (m >= 1 && m <= n) ? sg[(size_t)(m - 1) * T] * g.sc.u_scale : 0.0f;
                            }
                            *reinterpret_cast<uint4 *>(ug + chunk_off(row, c8 >> 3, c8 & 7)) =
                                make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
                        }
                    }
                }
                // the step's lambda_i(t_k) (every warp: it enters the bias) and C_i(t_k)
                for (int j = lane; j < n; j += 32) {
                    lw[j] = a.row[(size_t)k * n + j].x;
                    lw[npad + j] = g.Ctab[(size_t)k * n + j];
                }
                __syncwarp();
                // feature rows written and (after the previous step's last rate) the
                // accumulators free: the first rate's first-layer products may start
                fence_async_smem();
                tc_before();
                __syncwarp();
                if (lane == 0)
                    for (int gi = 0; gi < kGroups; ++gi) mbar_arrive(&opu[gi]);
                const float xt_b = bf16_round(xt);
                // half first-layer bias of rate r for this warp's 32 columns, into slot r & 1:
                // (b_0 + W_0[:, t] t + W_0[:, i] r + W_0[:, lambda] lambda_r) / 2, the inputs
                // rounded to BF16 as the feature row would hold them
                auto rate_bias = [&](int r) {
                    const float xi_b = bf16_round((float)r * g.sc.i_scale);
                    const float xl_b = bf16_round(lw[r - 1] * g.sc.lam_scale);
                    const int c = cq * 32 + lane;
                    hbw[(r & 1) * 32 + lane] =
                        fmaf(w0c[2 * kH + c], xl_b, fmaf(w0c[kH + c], xi_b, fmaf(w0c[c], xt_b, bias[c])));
                    __syncwarp();
                };
                // Euler step of rate r for this row's path in tile gi with A_r = C_r + s_y f;
                // the owner applies it one rate late, off the products' critical path
                float pend_own[kGroups] = {0.0f, 0.0f};
                auto euler = [&](int r, int gi) {
                    if (!warp_wait(&outb[gi], pho[gi], abort, g.err)) return false;
                    pho[gi] ^= 1;
                    const float *op = opart + (size_t)gi * 3 * kRows + row;
                    const float o = pend_own[gi] + op[0] + op[kRows] + op[2 * kRows];
                    const float A = lw[npad + r - 1] + g.sc.y_scale * (o + b_out);
                    float *sp = st + (size_t)(r - 1) * T + gi * kRows;
                    const float z = sp[0] + fmaf(lw[r - 1], dH[gi], -A * h);
                    sp[0] = z;
                    if (mat && sidx[gi] != ~0ull)
                        a.snap[((size_t)(imin - 1) * n + (r - 1)) * a.snap_pitch + sidx[gi]] = z + a.Z0[r - 1];
                    return true;
                };
                rate_bias(n);
                for (int i = n; ok && i >= imin; --i) {
                    const float *hb0 = hbw + (i & 1) * 32;
#pragma unroll
                    for (int l = 0; l < L; ++l) {
#pragma unroll
                        for (int gi = 0; gi < kGroups; ++gi) {
                            if (!ok) continue;
                            if (!warp_wait(&dnb[gi], phd[gi], abort, g.err)) { ok = false; continue; }
                            phd[gi] ^= 1;
                            tc_after();
                            const uint32_t dbuf = dq + gi * kH;
                            const float *hbl = l == 0 ? hb0 : bias + l * kH + cq * 32;
                            float o4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                            uint32_t ra[16], rb[16];
                            tmem_ld16(dbuf, ra);
                            tmem_wait(ra);
                            tmem_ld16(dbuf + 16, rb);
#pragma unroll
                            for (int cc = 0; cc < 2; ++cc) {
                                // columns 32 cq + 16 cc .. +15; the second chunk loads meanwhile
                                uint32_t(&cur)[16] = cc ? rb : ra;
                                uint32_t pk[8];
#pragma unroll
                                for (int qd = 0; qd < 2; ++qd) {
                                    float sv[8];
                                    silu8(cur + qd * 8, hbl + cc * 16 + qd * 8, sv);
                                    if (l < L - 1) {
#pragma unroll
                                        for (int e = 0; e < 4; ++e) pk[qd * 4 + e] = pack2(sv[2 * e], sv[2 * e + 1]);
                                    } else {
                                        const float4 w0 = *reinterpret_cast<const float4 *>(wout + cq * 32 + cc * 16 + qd * 8);
                                        const float4 w1 = *reinterpret_cast<const float4 *>(wout + cq * 32 + cc * 16 + qd * 8 + 4);
                                        const float wo[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                                        for (int e = 0; e < 8; e += 2) {
                                            // BF16 activations (packed round to nearest even), FP32 products
                                            const uint32_t pk = pack2(sv[e], sv[e + 1]);
                                            o4[e & 3] = fmaf(__uint_as_float(pk << 16), wo[e], o4[e & 3]);
                                            o4[(e + 1) & 3] = fmaf(__uint_as_float(pk & 0xffff0000u), wo[e + 1], o4[(e + 1) & 3]);
                                        }
                                    }
                                }
                                // activations K = 32 cq + 16 cc .. +15 of this row: 8 packed TMEM columns
                                if (l < L - 1) tmem_st8(aq + gi * (kH / 2) + cc * 8, pk);
                                if (cc == 0) tmem_wait(rb);
                            }
                            if (l < L - 1) {
                                tmem_wait_st();
                                tc_before();
                                __syncwarp();
                                // the previous rate's Euler step: its output partials can be
                                // overwritten only after this warp's next arrival on opx, or,
                                // with one hidden product per rate, after this one
                                if (l == 0 && owner && i < n && L == 2)
                                    if (!euler(i + 1, gi)) { ok = false; continue; }
                                if (lane == 0) mbar_arrive(&opx[gi]);
                                if (l == 0 && owner && i < n && L > 2)
                                    if (!euler(i + 1, gi)) { ok = false; continue; }
                                if (l == 0 && gi == kGroups - 1 && i > imin) rate_bias(i - 1);
                            } else {
                                // this tile's accumulator has been read: the next rate's
                                // first-layer product may overwrite it (after the last
                                // rate, the next step's feature rows come first)
                                tc_before();
                                __syncwarp();
                                if (lane == 0 && i > imin) mbar_arrive(&opu[gi]);
                                const float part = (o4[0] + o4[1]) + (o4[2] + o4[3]);
                                if (owner) {
                                    pend_own[gi] = part;
                                } else {
                                    opart[((size_t)gi * 3 + (cq - 1)) * kRows + row] = part;
                                    __syncwarp();
                                    if (lane == 0) mbar_arrive(&outb[gi]);
                                }
                            }
                        }
                    }
                }
                // the step's last rate
                if (owner)
                    for (int gi = 0; ok && gi < kGroups; ++gi)
                        if (!euler(imin, gi)) ok = false;
                if (!ok) break;
                if (mat && owner) {
                    // the 4 owner warps reduce their paths of both tiles; the first of
                    // them adds the four sums in fixed order
                    const int m = imin, buf = mcount & 1;
                    ++mcount;
                    double Pp[kGroups], Sp[kGroups];
                    float Lm[kGroups];
#pragma unroll
                    for (int gi = 0; gi < kGroups; ++gi)
                        maturity_products(a, m, [&](int i) { return st[(size_t)(i - 1) * T + gi * kRows] + a.Z0[i - 1]; },
                                          Pp[gi], Sp[gi], Lm[gi]);
                    for (int qs = 0; qs < ns; ++qs) {
                        const float K = a.strikes[(size_t)(m - 1) * ns + qs];
                        const size_t slot = ((size_t)buf * 4 + q4) * ns + qs;
                        if (a.product == 0) {
                            float v[kGroups];
#pragma unroll
                            for (int gi = 0; gi < kGroups; ++gi)
                                v[gi] = active[gi] ? caplet_payoff(a, (float)Pp[gi], Lm[gi], K) : 0.0f;
                            const float4 r = caplet_warp_sums(v);
                            if (lane == 0) reinterpret_cast<float4 *>(red)[slot] = r;
                            continue;
                        }
                        double s1 = 0.0, s2 = 0.0;
#pragma unroll
                        for (int gi = 0; gi < kGroups; ++gi) {
                            const double pay = active[gi] ? payoff(a, Pp[gi], Sp[gi], Lm[gi], K) : 0.0;
                            s1 += pay;
                            s2 += pay * pay;
                        }
                        s1 = warp_sum(s1);
                        s2 = warp_sum(s2);
                        if (lane == 0) {
                            red[2 * slot + 0] = s1;
                            red[2 * slot + 1] = s2;
                        }
                    }
                    if (lane == 0) mbar_arrive(&payb[0]);
                    if (q4 == 0) {
                        if (!warp_wait(&payb[0], php, abort, g.err)) { ok = false; break; }
                        for (int qs = lane; qs < ns; qs += 32) { // one strike per lane
                            double s1, s2;
                            block_payoff_sums(a, red + (size_t)buf * 4 * ns * 2, 4, ns, qs, s1, s2);
                            double *acc = bsum + 4 * ((size_t)(m - 1) * ns + qs);
                            kahan_add(acc + 0, acc + 1, s1);
                            kahan_add(acc + 2, acc + 3, s2);
                        }
                    }
                    php ^= 1;
                }
            }
        }
    }
    tc_before();
    __syncthreads();
    if (warp == kEpiWarps) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGroups * 2 * kH));
    }
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += kThreads) {
        out[2 * e + 0] = bsum[4 * e + 0];
        out[2 * e + 1] = bsum[4 * e + 2];
    }
}


// ---------------------------------------------------------------------------
// Vector head: one network pass per (path, Euler step) gives every rate's
// compensator.  The CTA layout is the per-rate kernel's (two tiles of 128
// paths, sixteen epilogue warps shared by both tiles, activations in TMEM, one
// MMA lane).  W_out's rows are staged two columns down, so that output column c
// belongs to rate c - 1, the rate whose log-rate sits in feature column c: the
// warp of column quarter cq reads its 16 output columns (chunks cq and cq + 4),
// applies the Euler step of those rates and writes their feature columns for
// the next step, with no exchange between warps.
// ---------------------------------------------------------------------------
constexpr int kOut = 48;                       // network outputs (column i - 1 for rate i; n <= 48)
constexpr int kOutN = 64;                      // output product width: columns 0 .. 63, rate c - 1
constexpr int kOutBlock = kOutN * 128;         // one 64-wide K block of the staged W_out

struct TcVecLayout {
    uint32_t w0, w, wo, u, bias, bout, bars, misc, red, bsum, state, lc, dh, total;
};

__host__ __device__ inline TcVecLayout tc_vec_layout(int L, int KB0, int n, int ns)
{
    TcVecLayout t;
    uint32_t o = 0;
    t.w0 = o; o += KB0 * kTileBytes;             // W_0: H rows x 64 KB0 columns
    t.w = o; o += (L - 1) * 2 * kTileBytes;       // W_1 .. W_{L-1}
    t.wo = o; o += 2 * kOutBlock;                 // W_out staged: 64 rows x 128 columns
    t.u = o; o += kGroups * KB0 * kTileBytes;     // feature rows, per tile
    t.bias = o; o += L * kH * 4;                  // b_0 / 2 .. b_{L-1} / 2
    t.bout = o; o += kOutN * 4;                   // output bias of column c (rate c - 1)
    t.bars = o; o += 12 * 8;                      // mbarriers
    t.misc = o; o += 16;                          // TMEM base, abort word
    o = (o + 15) & ~15u;
    t.red = o; o += 2 * 4 * ns * 2 * 8;           // 4 owner warps' payoff sums, two buffers
    t.bsum = o; o += n * ns * 4 * 8;              // Kahan accumulators
    t.state = o; o += n * kGroups * kRows * 4;    // log-rate offsets of the CTA's paths, [rate][path]
    t.lc = o; o += kEpiWarps * 2 * 16 * 4;        // per warp: lambda and C of its 16 rates at t_k
    t.dh = o; o += 2 * kGroups * kRows * 4;       // increments of the CTA's paths, two steps
    t.total = o + 1024;                           // slack for aligning the base
    return t;
}

template <int L, int KB0>
__global__ void __launch_bounds__(kThreads, 1) mlp_tc_vec_kernel(const PathArgs a, const MlpArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    const int n = a.n, s = a.s, S = a.S, ns = a.ns;
    const TcVecLayout lay = tc_vec_layout(L, KB0, n, ns);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = saddr(sm);
    float *bias = reinterpret_cast<float *>(sm + lay.bias);
    float *bout = reinterpret_cast<float *>(sm + lay.bout);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + lay.bars);
    uint64_t *opu = bars + 0;   // [kGroups] feature rows written, accumulator free (every epilogue warp)
    uint64_t *opx = bars + 2;   // [kGroups] activations written (every epilogue warp)
    uint64_t *dnb = bars + 4;   // [kGroups] product complete (commit)
    uint64_t *eul = bars + 6;   // Euler steps of quarters 1..3 done, at a maturity (12 warps)
    uint64_t *payb = bars + 7;  // payoff partials written (the 4 path-owning warps)
    uint64_t *finb = bars + 8;  // all products complete (commit)
    uint64_t *dhb = bars + 9;   // [2] a step's increments written (quarters 2 and 3, one tile each), by step parity
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + lay.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + lay.misc + 4);
    double *red = reinterpret_cast<double *>(sm + lay.red);
    double *bsum = reinterpret_cast<double *>(sm + lay.bsum);
    const int in_pad = g.in_pad;

    // weights into the swizzled operand layout; W_out row j (rate j + 1) goes to row j + 2
    for (int l = 0; l <= L; ++l) {
        const int din = l == 0 ? in_pad : kH;
        const int rows = l == L ? kOutN : kH;
        const int chunks = l == 0 ? KB0 * 8 : 16;
        const uint32_t base = l == 0 ? lay.w0 : (l == L ? lay.wo : lay.w + (l - 1) * 2 * kTileBytes);
        for (int e = tid; e < rows * chunks; e += kThreads) {
            const int h = e / chunks, c = e % chunks;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (l < L) {
                if (c * 8 < din) v = *reinterpret_cast<const uint4 *>(g.wh + g.offW[l] + (size_t)h * din + c * 8);
            } else if (h >= 2 && h - 2 < kOut) {
                v = *reinterpret_cast<const uint4 *>(g.wh + g.off_wout + (size_t)(h - 2) * din + c * 8);
            }
            *reinterpret_cast<uint4 *>(sm + base + (c >> 3) * rows * 128 + (h >> 3) * 1024 + (h & 7) * 128 +
                                       (((c & 7) ^ (h & 7)) << 4)) = v;
        }
    }
    for (int e = tid; e < L * kH; e += kThreads) bias[e] = 0.5f * g.wp[g.offb[e / kH] + e % kH];
    for (int e = tid; e < kOutN; e += kThreads) bout[e] = (e >= 2 && e - 2 < kOut) ? g.wp[g.off_bout + e - 2] : 0.0f;
    for (int e = tid; e < 4 * n * ns; e += kThreads) bsum[e] = 0.0;
    if (tid == 0) {
        for (int gi = 0; gi < kGroups; ++gi) {
            mbar_init(&opu[gi], kEpiWarps);
            mbar_init(&opx[gi], kEpiWarps);
            mbar_init(&dnb[gi], 1);
        }
        mbar_init(eul, 12);
        mbar_init(payb, 4);
        mbar_init(finb, 1);
        mbar_init(&dhb[0], 4 * kGroups);
        mbar_init(&dhb[1], 4 * kGroups);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(4 * kH));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot; // accumulator of tile gi: columns [128 gi, +128); activations [256 + 64 gi, +64)
    const int T = kGroups * kRows;
    const uint64_t ntiles = (a.paths + T - 1) / T;

    if (warp == kEpiWarps) {
        // MMA issuer: per step and tile, the first layer (feature rows), the
        // hidden layers and the output product (activations in TMEM), tiles in turn
        if (lane == 0) {
            uint32_t phu = 0, phx = 0; // bit gi: phase parity of opu[gi], opx[gi]
            bool ok = !g.stall_mma;
            for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x)
                for (int k = 0; ok && k < S; ++k)
                    for (int l = 0; ok && l <= L; ++l)
                        for (int gi = 0; gi < kGroups; ++gi) {
                            uint64_t *ob = l == 0 ? &opu[gi] : &opx[gi];
                            uint32_t &ph = l == 0 ? phu : phx;
                            if (!mbar_wait(ob, (ph >> gi) & 1u, abort, g.err)) { ok = false; break; }
                            ph ^= 1u << gi;
                            tc_after();
                            const uint32_t d = tmem + gi * kH;
                            if (l == 0) {
                                const uint32_t abase = sbase + lay.u + gi * KB0 * kTileBytes;
                                for (int ks = 0; ks < in_pad / 16; ++ks) {
                                    const uint32_t off = (ks >> 2) * kTileBytes + (ks & 3) * 32;
                                    mma_bf16(d, sdesc(abase + off), sdesc(sbase + lay.w0 + off), ks > 0);
                                }
                            } else {
                                const uint32_t at = tmem + 2 * kH + gi * (kH / 2);
                                const uint32_t bbase = sbase + (l == L ? lay.wo : lay.w + (l - 1) * 2 * kTileBytes);
                                const uint32_t bstride = l == L ? (uint32_t)kOutBlock : (uint32_t)kTileBytes;
                                const uint32_t id = l == L ? idesc_n(kOutN) : kIdesc;
                                for (int ks = 0; ks < kH / 16; ++ks) {
                                    const uint32_t bo = (ks >> 2) * bstride + (ks & 3) * 32;
                                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                                                 ::"r"(d), "r"(at + ks * 8), "l"(sdesc(bbase + bo)), "r"(id),
                                                 "r"((uint32_t)(ks > 0)));
                                }
                            }
                            mma_commit(&dnb[gi]);
                        }
            mma_commit(finb);
            volatile int dummy_abort = 0;
            mbar_wait(finb, 0, &dummy_abort, g.err);
        }
        __syncwarp();
    } else {
        // warp = 4 cq + q4: TMEM lane quadrant q4 (row 32 q4 + lane of each tile) and
        // column quarter cq: columns 32 cq .. +31 of the hidden layers; output and
        // feature columns 8 cq .. +7 and 8 cq + 32 .. +39 (chunks cq and cq + 4, so
        // that the live rates spread evenly), that is rates column - 1.
        const int cq = warp >> 2, q4 = warp & 3;
        const int row = q4 * 32 + lane;
        const bool owner = cq == 0;
        // output / feature column of this warp's c-th rate (c = 0 .. 15)
        auto col_of = [&](int c) { return (c < 8 ? 8 * cq : 8 * cq + 24) + c; };
        const uint32_t dq = tmem + ((uint32_t)(q4 * 32) << 16);
        float *st = reinterpret_cast<float *>(sm + lay.state) + row; // [rate][path]: + (m - 1) T + gi * kRows
        float *lw = reinterpret_cast<float *>(sm + lay.lc) + warp * 32; // lambda, C of this warp's 16 rates
        const float h = a.h;
        uint32_t phd = 0, php = 0, phe = 0, phh = 0; // bit gi: phase parity of dnb[gi]; bit b: of dhb[b]
        int mcount = 0;
        uint64_t gstep = 0; // steps begun by this CTA: a step's increments live in buffer gstep & 1
        float *dhs = reinterpret_cast<float *>(sm + lay.dh) + row; // [buffer][tile][row]
        bool ok = true;
        // feature chunks 2 cq, 2 cq + 1 of the row at time index k: column c holds t
        // (c = 0), u_0 = 0 (c = 1) or u_{c-1} s_u
        auto write_features = [&](int k, int gi) {
            const float xt = (float)k * h * g.sc.t_scale;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c8 = cq + 4 * q;
                if (c8 >= KB0 * 8) continue;
                float f[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int c = c8 * 8 + e, m = c - 1;
                    f[e] = c == 0 ? xt : ((m >= 1 && m <= n) ? st[(size_t)(m - 1) * T + gi * kRows] * g.sc.u_scale : 0.0f);
                }
                *reinterpret_cast<uint4 *>(sm + lay.u + gi * KB0 * kTileBytes + chunk_off(row, c8 >> 3, c8 & 7)) =
                    make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
            }
        };
        for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            const uint64_t lp0 = tile * (uint64_t)T + row; // + gi * kRows
            if (!owner && mcount > 0) {
                // the owners price the previous tiles' last maturity from every rate's
                // state: wait for their payoff partials before resetting this warp's rates
                if (!warp_wait(payb, (uint32_t)((mcount - 1) & 1), abort, g.err)) { ok = false; break; }
            }
            for (int c = 0; c < 16; ++c) {
                const int m = col_of(c) - 1;
                if (m >= 1 && m <= n)
#pragma unroll
                    for (int gi = 0; gi < kGroups; ++gi) st[(size_t)(m - 1) * T + gi * kRows] = 0.0f;
            }
            for (int gi = 0; gi < kGroups; ++gi) write_features(0, gi);
            fence_async_smem();
            tc_before();
            __syncwarp();
            if (lane == 0)
                for (int gi = 0; gi < kGroups; ++gi) mbar_arrive(&opu[gi]);
            // each step's increments are drawn once, tile gi by the warps of column
            // quarter 2 + gi, and shared with the others (two buffers and barriers,
            // alternating by step)
            auto draw_share = [&](int kk, int b) {
                const int gi = cq - (4 - kGroups);
                dhs[(b * kGroups + gi) * kRows] = draw_increment(a, a.first_path + lp0 + gi * kRows, (uint32_t)kk);
                __syncwarp();
                if (lane == 0) mbar_arrive(&dhb[b]);
            };
            const bool drawer = cq >= 4 - kGroups; // quarters 2 and 3: the fewest low-index rates
            if (drawer) draw_share(0, (int)(gstep & 1));
            // this warp's rates' lambda and C, loaded one step ahead of their use
            const int mine = lane < 16 ? col_of(lane) - 1 : 0;
            const bool in = lane < 16 && mine >= 1 && mine <= n;
            float lam_next = in ? a.row[mine - 1].x : 0.0f, c_next = in ? g.Ctab[mine - 1] : 0.0f;
            for (int k = 0; ok && k < S; ++k) {
                const int imin = k / s + 1;
                const bool mat = (k + 1) % s == 0;
                const int gb = (int)(gstep++ & 1);
                if (lane < 16) {
                    lw[lane] = lam_next;
                    lw[16 + lane] = c_next;
                }
                __syncwarp();
                if (in && k + 1 < S) {
                    lam_next = a.row[(size_t)(k + 1) * n + (mine - 1)].x;
                    c_next = g.Ctab[(size_t)(k + 1) * n + (mine - 1)];
                }
                // hidden layers: SiLU of 32 columns, BF16 activations into TMEM
#pragma unroll
                for (int l = 0; l < L; ++l) {
#pragma unroll
                    for (int gi = 0; gi < kGroups; ++gi) {
                        if (!ok) continue;
                        if (!warp_wait(&dnb[gi], (phd >> gi) & 1u, abort, g.err)) { ok = false; continue; }
                        phd ^= 1u << gi;
                        tc_after();
                        const uint32_t dbuf = dq + gi * kH + cq * 32;
                        const float *hbl = bias + l * kH + cq * 32;
                        uint32_t ra[16], rb[16];
                        tmem_ld16(dbuf, ra);
                        tmem_wait(ra);
                        tmem_ld16(dbuf + 16, rb);
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc) {
                            uint32_t(&cur)[16] = cc ? rb : ra;
                            uint32_t pk[8];
#pragma unroll
                            for (int qd = 0; qd < 2; ++qd) {
                                float sv[8];
                                silu8(cur + qd * 8, hbl + cc * 16 + qd * 8, sv);
#pragma unroll
                                for (int e = 0; e < 4; ++e) pk[qd * 4 + e] = pack2(sv[2 * e], sv[2 * e + 1]);
                            }
                            tmem_st8(dq + 2 * kH + gi * (kH / 2) + cq * 16 + cc * 8, pk);
                            if (cc == 0) tmem_wait(rb);
                        }
                        tmem_wait_st();
                        tc_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&opx[gi]);
                    }
                }
                // output product: this warp's 16 rates, Euler step and next feature columns
                if (ok) {
                    if (!warp_wait(&dhb[gb], (phh >> gb) & 1u, abort, g.err)) ok = false;
                    phh ^= 1u << gb;
                }
                float dH[kGroups];
#pragma unroll
                for (int gi = 0; gi < kGroups; ++gi) dH[gi] = dhs[(gb * kGroups + gi) * kRows];
#pragma unroll
                for (int gi = 0; gi < kGroups; ++gi) {
                    if (!ok) continue;
                    if (!warp_wait(&dnb[gi], (phd >> gi) & 1u, abort, g.err)) { ok = false; continue; }
                    phd ^= 1u << gi;
                    tc_after();
                    uint32_t ro[16];
                    tmem_ld8(dq + gi * kH + 8 * cq, ro);
                    tmem_ld8(dq + gi * kH + 8 * cq + 32, ro + 8);
                    tmem_wait(ro);
                    const uint64_t lp = lp0 + gi * kRows;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int m = col_of(c) - 1;
                        if (m < imin || m > n) continue; // also m < 1: imin >= 1
                        const float f = __uint_as_float(ro[c]) + bout[col_of(c)];
                        const float A = lw[16 + c] + g.sc.y_scale * f;
                        float *sp = st + (size_t)(m - 1) * T + gi * kRows;
                        const float z = sp[0] + fmaf(lw[c], dH[gi], -A * h);
                        sp[0] = z;
                        if (mat && a.snap != nullptr && lp < a.paths && lp % a.snap_stride == 0 &&
                            lp / a.snap_stride < a.n_snap)
                            a.snap[((size_t)(imin - 1) * n + (m - 1)) * a.snap_pitch + lp / a.snap_stride] = z + a.Z0[m - 1];
                    }
                }
                if (!ok) break;
                // next step's feature columns of these rates; accumulators read
                if (k + 1 < S) {
                    for (int gi = 0; gi < kGroups; ++gi) write_features(k + 1, gi);
                    fence_async_smem();
                    tc_before();
                    __syncwarp();
                    if (lane == 0)
                        for (int gi = 0; gi < kGroups; ++gi) mbar_arrive(&opu[gi]);
                    if (drawer) draw_share(k + 1, (int)(gstep & 1));
                } else {
                    tc_before();
                }
                if (mat) {
                    // the owner warps price with every rate of the row's paths
                    if (!owner) {
                        __syncwarp();
                        if (lane == 0) mbar_arrive(eul);
                        ++mcount; // the owners' payoff phases, counted alike
                        continue;
                    }
                    if (!warp_wait(eul, phe, abort, g.err)) { ok = false; break; }
                    phe ^= 1;
                    const int m = imin, buf = mcount & 1;
                    ++mcount;
                    double Pp[kGroups], Sp[kGroups];
                    float Lm[kGroups];
#pragma unroll
                    for (int gi = 0; gi < kGroups; ++gi)
                        maturity_products_grouped(a, m, [&](int i) { return st[(size_t)(i - 1) * T + gi * kRows] + __ldg(a.Z0 + i - 1); },
                                                  Pp[gi], Sp[gi], Lm[gi]);
                    for (int qs = 0; qs < ns; ++qs) {
                        const float K = a.strikes[(size_t)(m - 1) * ns + qs];
                        const size_t slot = ((size_t)buf * 4 + q4) * ns + qs;
                        if (a.product == 0) {
                            float v[kGroups];
#pragma unroll
                            for (int gi = 0; gi < kGroups; ++gi)
                                v[gi] = lp0 + gi * kRows < a.paths ? caplet_payoff(a, (float)Pp[gi], Lm[gi], K) : 0.0f;
                            const float4 r = caplet_warp_sums(v);
                            if (lane == 0) reinterpret_cast<float4 *>(red)[slot] = r;
                            continue;
                        }
                        double s1 = 0.0, s2 = 0.0;
#pragma unroll
                        for (int gi = 0; gi < kGroups; ++gi) {
                            const double pay = lp0 + gi * kRows < a.paths ? payoff(a, Pp[gi], Sp[gi], Lm[gi], K) : 0.0;
                            s1 += pay;
                            s2 += pay * pay;
                        }
                        s1 = warp_sum(s1);
                        s2 = warp_sum(s2);
                        if (lane == 0) {
                            red[2 * slot + 0] = s1;
                            red[2 * slot + 1] = s2;
                        }
                    }
                    if (lane == 0) mbar_arrive(payb);
                    if (q4 == 0) {
                        if (!warp_wait(payb, php, abort, g.err)) { ok = false; break; }
                        for (int qs = lane; qs < ns; qs += 32) { // one strike per lane
                            double s1, s2;
                            block_payoff_sums(a, red + (size_t)buf * 4 * ns * 2, 4, ns, qs, s1, s2);
                            double *acc = bsum + 4 * ((size_t)(m - 1) * ns + qs);
                            kahan_add(acc + 0, acc + 1, s1);
                            kahan_add(acc + 2, acc + 3, s2);
                        }
                    }
                    php ^= 1;
                }
            }
        }
    }
    tc_before();
    __syncthreads();
    if (warp == kEpiWarps) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * kH));
    }
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += kThreads) {
        out[2 * e + 0] = bsum[4 * e + 0];
        out[2 * e + 1] = bsum[4 * e + 2];
    }
}

typedef void (*TcKernelFn)(const PathArgs, const MlpArgs);

TcKernelFn pick_tc(int L, int KB0)
{
    if (KB0 == 1) {
        switch (L) {
        case 2: return mlp_tc_kernel<2, 1>;
        case 3: return mlp_tc_kernel<3, 1>;
        case 4: return mlp_tc_kernel<4, 1>;
        default: return nullptr;
        }
    }
    if (KB0 == 2) {
        switch (L) {
        case 2: return mlp_tc_kernel<2, 2>;
        default: return nullptr;
        }
    }
    return nullptr;
}

TcKernelFn pick_tc_vec(int L, int KB0)
{
    if (KB0 != 1) return nullptr;
    switch (L) {
    case 2: return mlp_tc_vec_kernel<2, 1>;
    case 3: return mlp_tc_vec_kernel<3, 1>;
    case 4: return mlp_tc_vec_kernel<4, 1>;
    default: return nullptr;
    }
}

}  // namespace

size_t mlp_tc_vec_smem(int layers, int in_pad, int n, int ns)
{
    return tc_vec_layout(layers, (in_pad + 63) / 64, n, ns).total;
}

bool mlp_tc_vec_supported(int hidden, int layers, int in_pad, int outputs, int n)
{
    return hidden == kH && outputs == kOut && n <= kOut && in_pad % 16 == 0 &&
           pick_tc_vec(layers, (in_pad + 63) / 64) != nullptr;
}

int mlp_tc_vec_occupancy(int layers, int in_pad, size_t smem, int *blocks_per_sm)
{
    TcKernelFn f = pick_tc_vec(layers, (in_pad + 63) / 64);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem);
}

int launch_mlp_tc_vec(int layers, int in_pad, int grid, size_t smem, cudaStream_t st, const PathArgs &a,
                      const MlpArgs &g)
{
    TcKernelFn f = pick_tc_vec(layers, (in_pad + 63) / 64);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, kThreads, smem, st>>>(a, g);
    return (int)cudaGetLastError();
}

int mlp_tc_threads() { return kThreads; }
int mlp_tc_paths_per_block() { return kGroups * kRows; }

size_t mlp_tc_smem(int layers, int in_pad, int n, int ns)
{
    return tc_layout(layers, (in_pad + 63) / 64, n, ns).total;
}

bool mlp_tc_supported(int hidden, int layers, int in_pad)
{
    return hidden == kH && in_pad % 16 == 0 && pick_tc(layers, (in_pad + 63) / 64) != nullptr;
}

int mlp_tc_occupancy(int layers, int in_pad, size_t smem, int *blocks_per_sm)
{
    TcKernelFn f = pick_tc(layers, (in_pad + 63) / 64);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem);
}

int launch_mlp_tc(int layers, int in_pad, int grid, size_t smem, cudaStream_t st, const PathArgs &a,
                  const MlpArgs &g)
{
    TcKernelFn f = pick_tc(layers, (in_pad + 63) / 64);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, kThreads, smem, st>>>(a, g);
    return (int)cudaGetLastError();
}

}  // namespace lll
