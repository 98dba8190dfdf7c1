// lll_mlp_wide.cu -- the full scheme with the learned compensator (LLL_MLP)
// for a vector-head network of width 256 (the N = 120 network, input
// (t, u_0 .. u_{N-1}), four hidden layers, one output per rate), the whole
// simulation in one persistent kernel on the 5th-generation tensor cores.
//
// Method (the same as the layer-by-layer scheme of lll_mlp_layered.cu and the
// fused kernels of lll_mlp_tc.cu): Euler steps of Eq. (log-LIB-SDE-2) with the
// drift of Eq. (LIBOR-drift-PT), the jump compensator of every live rate being
// A_i = C_i + s_y f_i(x), where x = (t s_t, u_0, u_1 s_u, .., u_n s_u) holds
// the log-rate offsets of the path at t_k and f is the trained network
// (SiLU hidden layers, BF16 weights and activations, FP32 accumulation);
// caplet (or co-terminal swaption) payoffs at every T_m, Eq. (caplet).
//
// A CTA owns a tile of 128 paths (one per TMEM lane) for all S Euler steps,
// then takes the next tile.  Per step the network runs layer after layer on
// the tile: activations [128 x 256] BF16 stay in shared memory (four 64-wide
// K blocks, 128-byte swizzled K-major: the A operand), the weights stream
// from L2 through a three-stage ring of 64-wide K blocks (TMA, the B
// operand), and the products accumulate FP32 into one of two 256-column
// tensor-memory accumulators, alternating by layer, so that the products of
// layer l + 1 start on the first K block of layer l's activations while the
// epilogue is still writing the rest.
// Roles (576 threads):
//  * warps 0-15, epilogue: warp 4 cq + q4 reads TMEM lane quadrant q4 (paths
//    32 q4 .. + 31).  Hidden layer: per K block j it reads accumulator
//    columns 64 j + 16 cq .. + 15, adds the bias, applies SiLU and writes the
//    two BF16 chunks into activation block j, then arrives on block j's
//    barrier.  Output layer: it reads output chunks cq + 4 i (i = 0..3), so
//    that live rates stay spread over the warps as the low rates expire,
//    applies the Euler step to those rates (state [rate][path] in shared
//    memory) and writes the same chunks of the next step's feature row.
//    Output and feature column c belong to rate c - 1 (the output layer's
//    weight rows are loaded two rows down).  Each step's increments, and the
//    step's table of lambda and -h (C + s_y b_out) per column, are written
//    by the four warps of one column quarter, in turn.  At a caplet maturity
//    every warp multiplies the factors (1 + delta L_i) of its live rates past
//    the maturing one while it updates them; the warps of quarter 0 combine
//    the four products of their paths (for swaptions they form P and S from
//    the shared state in rate order), price, and quarter 0, quadrant 0 adds
//    the CTA's sums into its cells in global memory (FP64; one thread per
//    cell, tiles in order, so the sums are deterministic).
//  * warp 16, lane 0: TMA producer of the weight ring.
//  * warp 17: allocates the 512 TMEM columns; lane 0 issues the products.
// Every wait is bounded: on timeout the CTA sets an abort word and the
// launch's error word, every role leaves its loop, the TMA lane waits for
// its loads in flight, the MMA lane drains its products, and the tensor
// memory is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "lll_device.cuh"
#include "lll_internal.h"
#include "lll_mlp.h"
#include "lll_tc.cuh"

namespace lll {
namespace {

using namespace tc;

constexpr int kHW = 256;                          // hidden width
constexpr int kRowsW = 128;                       // paths per tile (TMEM lanes)
constexpr int kEpiW = 16;                         // epilogue warps
constexpr int kProdWarp = kEpiW;
constexpr int kMmaWarp = kEpiW + 1;
constexpr int kThreadsW = (kEpiW + 2) * 32;
constexpr int kStagesW = 3;                       // weight ring stages
constexpr uint32_t kActBlock = kRowsW * 128;      // one 64-wide K block of the activations
constexpr uint32_t kStageBytes = kHW * 128;       // one 64-wide K block of a 256-row weight
constexpr int kOutW = 128;                        // output product width (column c: rate c - 1)
constexpr uint32_t kOutStage = kOutW * 128;       // one 64-wide K block of the staged output weights
constexpr int kMaxLayersW = 4;
constexpr int kMaxStrikesW = 16;

struct WideMaps {
    CUtensorMap w[kMaxLayersW + 1]; // W_0 .. W_{L-1} (boxes 64 x 256), W_out (boxes 64 x 128)
};

// Shared-memory plan: every region at a fixed offset except the path state,
// which comes last (n rows of kRowsW floats), so that the addresses fold into
// constants.
struct WideLayout {
    static constexpr uint32_t act = 0;                              // activations / feature rows of the tile
    static constexpr uint32_t ring = act + 4 * kActBlock;           // weight K blocks
    static constexpr uint32_t dh = ring + kStagesW * kStageBytes;   // increments of two steps
    static constexpr uint32_t lampc = dh + 2 * kRowsW * 4;          // [2 steps][lambda, -h (C + s_y b_out)][128 columns]
    static constexpr uint32_t red = lampc + 2 * 2 * kOutW * 4;      // payoff sums of the four pricing warps
    static constexpr uint32_t mpart = red + 4 * kMaxStrikesW * 2 * 4; // maturity: quarters' products, L_m
    static constexpr uint32_t bars = mpart + 5 * kRowsW * 4;        // mbarriers
    static constexpr uint32_t misc = bars + 20 * 8;                 // TMEM base, abort word
    static constexpr uint32_t state = misc + 16;                    // log-rate offsets, [rate][path]
    uint32_t total;
};

__host__ __device__ inline WideLayout wide_layout(int n, int)
{
    WideLayout t;
    t.total = WideLayout::state + (uint32_t)n * kRowsW * 4;
    return t;
}

// SiLU of 16 accumulator values v with biases b: with hz = (v + b) / 2,
// SiLU(v + b) = hz + hz tanh(hz), the function of the training kernels.
// Results packed as 8 BF16 pairs.
__device__ __forceinline__ void silu16(const uint32_t *v, const float4 (&b4)[4], uint32_t *pk)
{
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
        const float4 q = b4[e >> 2];
        const float b0 = (e & 2) ? q.z : q.x, b1 = (e & 2) ? q.w : q.y;
        const float2 hz = __ffma2_rn(make_float2(__uint_as_float(v[e]), __uint_as_float(v[e + 1])),
                                     make_float2(0.5f, 0.5f), make_float2(0.5f * b0, 0.5f * b1));
        const float2 t = make_float2(tanh_approx(hz.x), tanh_approx(hz.y));
        const float2 r = __ffma2_rn(hz, t, hz);
        pk[e >> 1] = pack2(r.x, r.y);
    }
}

template <int L, int KB0>
__global__ void __launch_bounds__(kThreadsW, 1)
    mlp_wide_kernel(const PathArgs a, const MlpArgs g, const __grid_constant__ WideMaps maps, double *acc)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw;
    if (saddr(smem_raw) & 1023u) { // the operand layout needs a 1024-byte aligned base
        if (threadIdx.x == 0) atomicOr(g.err, 2);
        return;
    }
    const int n = a.n, s = a.s, S = a.S, ns = a.ns;
    const WideLayout lay = wide_layout(n, ns);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = saddr(sm);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + lay.bars);
    uint64_t *full = bars;       // [3] weight block landed (TMA bytes)
    uint64_t *empty = bars + 3;  // [3] weight block consumed (commit)
    uint64_t *actb = bars + 6;   // [4] activation / feature block written (16 epilogue warps)
    uint64_t *accb = bars + 10;  // [2] accumulator complete (commit)
    uint64_t *dhb = bars + 12;   // [2] a step's increments written (4 warps), by step parity
    uint64_t *eul = bars + 14;   // Euler step of a maturity step done (16 warps)
    uint64_t *payb = bars + 15;  // payoff sums written (4 pricing warps)
    uint64_t *fin = bars + 16;   // every product complete (commit)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + lay.misc);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + lay.misc + 4);
    const uint64_t ntiles = (a.paths + kRowsW - 1) / kRowsW;

    if (tid == 0) {
        for (int i = 0; i < kStagesW; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int j = 0; j < 4; ++j) mbar_init(&actb[j], kEpiW);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accb[b], 1);
            mbar_init(&dhb[b], 4);
        }
        mbar_init(eul, kEpiW);
        mbar_init(payb, 4);
        mbar_init(fin, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(tslot, 2 * kHW);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot; // accumulator b: columns [256 b, 256 b + 256)

    if (warp == kProdWarp) {
        // ---------------- weight ring: one TMA box per 64-wide K block ----------------
        if (lane == 0) {
            for (int l = 0; l <= L; ++l) tma_prefetch_map(&maps.w[l]);
            uint32_t it = 0; // loads issued
            bool ok = true;
            for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x)
                for (int k = 0; ok && k < S; ++k)
                    for (int l = 0; ok && l <= L; ++l) {
                        const int nkb = l == 0 ? KB0 : 4;
                        for (int j = 0; j < nkb; ++j, ++it) {
                            const int st = (int)(it % kStagesW);
                            const uint32_t u = it / kStagesW;
                            if (u >= 1 && !(ok = mbar_wait(&empty[st], (u - 1) & 1u, abort, g.err))) break;
                            mbar_expect_tx(&full[st], l == L ? kOutStage : kStageBytes);
                            // the output weights two rows down: row c of the block is W_out row c - 2
                            tma_load_2d(sbase + lay.ring + st * kStageBytes, &maps.w[l], 64 * j, l == L ? -2 : 0,
                                        &full[st]);
                        }
                    }
            // no load may still be writing shared memory when the CTA exits: wait for
            // the last load into each stage (load it' = st + kStagesW u', the largest
            // such it' below it)
            volatile int no_abort = 0;
            for (uint32_t st = 0; st < kStagesW && st < it; ++st)
                mbar_wait(&full[st], ((it - 1 - st) / kStagesW) & 1u, &no_abort, g.err);
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- products: layer after layer, K block after K block ----------------
        if (lane == 0) {
            uint32_t it = 0, gl = 0, actph = 0; // actph bit j: phase parity of actb[j]
            bool ok = !g.stall_mma;
            for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x)
                for (int k = 0; ok && k < S; ++k)
                    for (int l = 0; ok && l <= L; ++l, ++gl) {
                        const uint32_t d = tmem + (gl & 1u) * kHW;
                        const uint32_t id = idesc_m128(l == L ? kOutW : kHW);
                        const int nkb = l == 0 ? KB0 : 4;
                        for (int j = 0; j < nkb; ++j, ++it) {
                            if (!(ok = mbar_wait(&actb[j], (actph >> j) & 1u, abort, g.err))) break;
                            actph ^= 1u << j;
                            const int st = (int)(it % kStagesW);
                            if (!(ok = mbar_wait(&full[st], (it / kStagesW) & 1u, abort, g.err))) break;
                            tc_after();
                            const uint32_t ab = sbase + lay.act + j * kActBlock;
                            const uint32_t bb = sbase + lay.ring + st * kStageBytes;
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks)
                                mma_ss(d, sdesc(ab + ks * 32), sdesc(bb + ks * 32), id, (j | ks) ? 1u : 0u);
                            mma_commit(&empty[st]);
                        }
                        if (ok) mma_commit(&accb[gl & 1u]);
                    }
            mma_commit(fin);
            volatile int no_abort = 0;
            mbar_wait(fin, 0, &no_abort, g.err);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps ----------------
        const int q4 = warp & 3, cq = warp >> 2, row = 32 * q4 + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
        float *st = reinterpret_cast<float *>(sm + lay.state) + row; // rate m at st[(m - 1) kRowsW]
        float *dhs = reinterpret_cast<float *>(sm + lay.dh);
        float *red = reinterpret_cast<float *>(sm + lay.red);
        float *mpart = reinterpret_cast<float *>(sm + lay.mpart); // [5][kRowsW]: products of quarters 0..3, L_m
        float *lampc = reinterpret_cast<float *>(sm + lay.lampc);
        const float h = a.h;
        // output / feature column of this warp's c-th column (c = 0..31): chunks cq + 4 i
        auto col_of = [&](int c) { return 8 * (cq + 4 * (c >> 3)) + (c & 7); };
        const int myrate = col_of(lane) - 1; // lane c holds Z0 of column c's rate
        const float z0_r = (myrate >= 1 && myrate <= n) ? a.Z0[myrate - 1] : 0.0f;
        // a drawing warp also writes lambda and -h (C + s_y b_out) of column row's rate
        const int drate = row - 1;
        const bool din = drate >= 1 && drate <= n;
        const float dbout = din ? g.wp[g.off_bout + drate - 1] : 0.0f;
        // the first tile's feature row at t = 0: every column zero (t = 0, u = 0)
        auto first_features = [&]() {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c8 = cq + 4 * i;
                if (c8 < KB0 * 8)
                    *reinterpret_cast<uint4 *>(sm + lay.act + (c8 >> 3) * kActBlock + swz(row, c8 & 7)) =
                        make_uint4(0, 0, 0, 0);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0)
                for (int j = 0; j < KB0; ++j) mbar_arrive(&actb[j]);
        };
        // 16 biases of this warp's columns in K block j of hidden layer l
        auto load_bias = [&](int l, int j, float4 (&bv)[4]) {
            const float4 *bp = reinterpret_cast<const float4 *>(g.wp + g.offb[l] + 64 * j + 16 * cq);
#pragma unroll
            for (int e = 0; e < 4; ++e) bv[e] = __ldg(bp + e);
        };
        uint32_t accph = 0, dhph = 0, eph = 0, pph = 0, gl = 0, gs = 0;
        bool ok = true;
        if ((uint64_t)blockIdx.x < ntiles) first_features();
        for (uint64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            const uint64_t lp = tile * kRowsW + row;
            const bool active = lp < a.paths;
            uint64_t sidx = ~0ull;
            if (a.snap != nullptr && active && lp % a.snap_stride == 0 && lp / a.snap_stride < a.n_snap)
                sidx = lp / a.snap_stride;
            const bool last_tile = tile + gridDim.x >= ntiles;
            for (int k = 0; ok && k < S; ++k, ++gs) {
                const int imin = k / s + 1;
                const bool mat = (k + 1) % s == 0;
                const bool drawer = cq == (int)(gs & 3u);
                float dlam = 0.0f, dc = 0.0f;
                if (drawer && din) { // loaded here, stored after the first hidden layer
                    dlam = a.row[(size_t)k * n + drate - 1].x;
                    dc = g.Ctab[(size_t)k * n + drate - 1];
                }
                // ---- hidden layers: bias + SiLU, BF16 activations block by block ----
#pragma unroll 1
                for (int l = 0; l < L; ++l, ++gl) {
                    const uint32_t b = gl & 1u;
                    const uint32_t ta = tl + b * kHW + 16 * cq;
                    float4 bv[4]; // biases of the next block, loaded ahead of their use
                    load_bias(l, 0, bv);
                    if (!(ok = warp_wait(&accb[b], (accph >> b) & 1u, abort, g.err))) break;
                    accph ^= 1u << b;
                    tc_after();
                    uint32_t r[2][16];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if ((j & 1) == 0) {
                            tmem_ld16(ta + 64 * j, r[0]);
                            tmem_ld16(ta + 64 * (j + 1), r[1]);
                            tmem_wait32(r[0]);
                        }
                        uint32_t pk[8];
                        silu16(r[j & 1], bv, pk);
                        if (j < 3) load_bias(l, j + 1, bv);
                        unsigned char *blk = sm + lay.act + j * kActBlock;
                        *reinterpret_cast<uint4 *>(blk + swz(row, 2 * cq)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *reinterpret_cast<uint4 *>(blk + swz(row, 2 * cq + 1)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        fence_async_smem();
                        tc_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&actb[j]);
                    }
                    if (!ok) break;
                    if (l == 0 && drawer) {
                        // this step's increments of the quadrant's paths, and the Euler
                        // coefficients of 32 columns
                        dhs[(gs & 1u) * kRowsW + row] = draw_increment(a, a.first_path + lp, (uint32_t)k);
                        lampc[(gs & 1u) * 2 * kOutW + row] = dlam;
                        lampc[(gs & 1u) * 2 * kOutW + kOutW + row] = -h * (dc + g.sc.y_scale * dbout);
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&dhb[gs & 1u]);
                    }
                }
                if (!ok) break;
                // ---- output layer: Euler step of this warp's rates, next feature chunks ----
                const uint32_t b = gl & 1u;
                ++gl;
                if (!(ok = warp_wait(&accb[b], (accph >> b) & 1u, abort, g.err))) break;
                accph ^= 1u << b;
                tc_after();
                const uint32_t db = gs & 1u;
                if (!(ok = warp_wait(&dhb[db], (dhph >> db) & 1u, abort, g.err))) break;
                dhph ^= 1u << db;
                const float dH = dhs[db * kRowsW + row];
                // z <- z + lambda dH - A h with A = C + s_y (f + b_out): per column,
                // lambda and -h (C + s_y b_out) at t_k from the step's table
                const float nh_ys = -h * g.sc.y_scale;
                const float *lam_t = lampc + db * 2 * kOutW, *pc_t = lam_t + kOutW;
                // the chunks then hold the next step's features, or a new tile's (t = 0, u = 0)
                const bool feat = k + 1 < S || !last_tile;
                const bool fresh = k + 1 >= S;
                const float xt = fresh ? 0.0f : (float)(k + 1) * h * g.sc.t_scale;
                // caplets at a maturity: this warp's factor of the product over rates > imin
                const bool cap = mat && a.product == 0;
                float pw = 1.0f;
                // one chunk of 8 columns (rates 8 c8 - 1 .. 8 c8 + 6): MODE 0 every rate
                // live, 1 every rate valid and expired (state unchanged), 2 any mix
                auto chunk = [&](auto mode, const uint32_t *acc8, int c8, int i) {
                    constexpr int MODE = decltype(mode)::value;
                    float zn[8], lam8[8], pc8[8];
                    if (MODE != 1) {
                        const float4 l0 = *reinterpret_cast<const float4 *>(lam_t + 8 * c8);
                        const float4 l1 = *reinterpret_cast<const float4 *>(lam_t + 8 * c8 + 4);
                        const float4 p0 = *reinterpret_cast<const float4 *>(pc_t + 8 * c8);
                        const float4 p1 = *reinterpret_cast<const float4 *>(pc_t + 8 * c8 + 4);
                        lam8[0] = l0.x; lam8[1] = l0.y; lam8[2] = l0.z; lam8[3] = l0.w;
                        lam8[4] = l1.x; lam8[5] = l1.y; lam8[6] = l1.z; lam8[7] = l1.w;
                        pc8[0] = p0.x; pc8[1] = p0.y; pc8[2] = p0.z; pc8[3] = p0.w;
                        pc8[4] = p1.x; pc8[5] = p1.y; pc8[6] = p1.z; pc8[7] = p1.w;
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int m = 8 * c8 + e - 1; // the rate of column 8 c8 + e
                        const bool valid = MODE < 2 || (m >= 1 && m <= n);
                        const bool live = MODE == 0 || (MODE == 2 && valid && m >= imin);
                        const float zo = (valid && (MODE == 1 || k > 0)) ? st[(m - 1) * kRowsW] : 0.0f;
                        if (MODE == 1) {
                            zn[e] = zo;
                            continue;
                        }
                        const float z0 = mat ? __shfl_sync(0xffffffffu, z0_r, 8 * i + e) : 0.0f;
                        const float z = zo + fmaf(lam8[e], dH, fmaf(nh_ys, __uint_as_float(acc8[e]), pc8[e]));
                        zn[e] = live ? z : zo;
                        if (live) {
                            st[(m - 1) * kRowsW] = z;
                            if (mat && sidx != ~0ull)
                                a.snap[((size_t)(imin - 1) * n + (m - 1)) * a.snap_pitch + sidx] = z + z0;
                            if (cap) {
                                // L_i(T_m) of the maturing rate; (1 + delta L_i) of the later ones
                                const float Li = expf(z + z0);
                                if (m == imin) mpart[4 * kRowsW + row] = Li;
                                else pw *= fmaf(a.delta, Li, 1.0f);
                            }
                        }
                    }
                    if (feat && c8 < KB0 * 8) {
                        float f[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int c = 8 * c8 + e, m = c - 1;
                            const bool valid = MODE < 2 || (m >= 1 && m <= n);
                            f[e] = (MODE == 2 && c == 0) ? xt : ((!fresh && valid) ? zn[e] * g.sc.u_scale : 0.0f);
                        }
                        *reinterpret_cast<uint4 *>(sm + lay.act + (c8 >> 3) * kActBlock + swz(row, c8 & 7)) =
                            make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
                    }
                };
                uint32_t ro[2][8];
                tmem_ld8(tl + b * kHW + 8 * cq, ro[0]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c8 = cq + 4 * i;
                    tmem_wait8(ro[i & 1]); // chunk i landed; chunk i + 1 loads while i is processed
                    if (i < 3) tmem_ld8(tl + b * kHW + 8 * (c8 + 4), ro[(i + 1) & 1]);
                    const int mlo = 8 * c8 - 1, mhi = 8 * c8 + 6; // the chunk's rates
                    if (mlo >= 1 && mlo >= imin && mhi <= n) chunk(std::integral_constant<int, 0>{}, ro[i & 1], c8, i);
                    else if (mlo >= 1 && mhi < imin && mhi <= n) chunk(std::integral_constant<int, 1>{}, ro[i & 1], c8, i);
                    else if (mlo <= n || (feat && c8 < KB0 * 8)) chunk(std::integral_constant<int, 2>{}, ro[i & 1], c8, i);
                }
                // the accumulator has been read; the feature chunks are written
                if (feat) {
                    fence_async_smem();
                    tc_before();
                    __syncwarp();
                    if (lane == 0)
                        for (int j = 0; j < KB0; ++j) mbar_arrive(&actb[j]);
                } else {
                    tc_before();
                }
                if (mat) {
                    if (cap) mpart[cq * kRowsW + row] = pw;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(eul);
                    if (cq == 0) {
                        // price the quadrant's paths with every rate's state
                        if (!(ok = warp_wait(eul, eph, abort, g.err))) break;
                        const int m = imin;
                        double Pp = 1.0, Sp = 1.0;
                        float Lm, Pf = 1.0f;
                        if (cap) {
                            // the product over rates > m, quarters in order (each in column order)
                            Pf = mpart[row];
#pragma unroll
                            for (int w = 1; w < 4; ++w) Pf *= mpart[w * kRowsW + row];
                            Lm = mpart[4 * kRowsW + row];
                        } else {
                            maturity_products_grouped(
                                a, m, [&](int i) { return st[(i - 1) * kRowsW] + __ldg(a.Z0 + i - 1); }, Pp, Sp, Lm);
                        }
                        // per-path payoffs are FP32 values (caplets) or FP64 (swaptions);
                        // the warp's sums over its 32 paths are formed in FP32, whose
                        // tree of 5 additions adds at most 5 2^-24 of the sum of |terms|
                        // (FP64 arithmetic is scarce on this part), and every later sum
                        // is FP64
                        for (int q0 = 0; q0 < ns; q0 += 4) {
                            float s1[4], s2[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int q = q0 + u;
                                // caplets: delta B(0, T_N) P (L_m - K)^+ in FP32, the value
                                // payoff() forms (its FP64 return is this FP32 number)
                                const float K = q < ns ? a.strikes[(size_t)(m - 1) * ns + q] : 0.0f;
                                const float pay = !(q < ns && active) ? 0.0f
                                                  : cap ? a.dBN * Pf * fmaxf(Lm - K, 0.0f)
                                                        : (float)payoff(a, Pp, Sp, Lm, K);
                                s1[u] = pay;
                                s2[u] = pay * pay;
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    s1[u] += __shfl_down_sync(0xffffffffu, s1[u], o);
                                    s2[u] += __shfl_down_sync(0xffffffffu, s2[u], o);
                                }
                            if (lane == 0)
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                    if (q0 + u < ns) {
                                        red[(q4 * ns + q0 + u) * 2 + 0] = s1[u];
                                        red[(q4 * ns + q0 + u) * 2 + 1] = s2[u];
                                    }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(payb);
                        if (q4 == 0) {
                            if (!(ok = warp_wait(payb, pph, abort, g.err))) break;
                            if (lane < ns) {
                                double s1 = 0.0, s2 = 0.0;
                                for (int w = 0; w < 4; ++w) {
                                    s1 += (double)red[(w * ns + lane) * 2 + 0];
                                    s2 += (double)red[(w * ns + lane) * 2 + 1];
                                }
                                // one thread per cell adds the CTA's tiles in order (no
                                // value returned: the lane does not wait for the add)
                                double *cell = acc + 4 * (((size_t)blockIdx.x * n + (m - 1)) * ns + lane);
                                atomicAdd(cell + 0, s1);
                                atomicAdd(cell + 2, s2);
                            }
                            __syncwarp();
                        }
                    }
                    eph ^= 1u;
                    pph ^= 1u;
                }
            }
        }
    }
    tc_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_after();
        tmem_dealloc(tmem, 2 * kHW);
    }
}

typedef void (*WideFn)(const PathArgs, const MlpArgs, const WideMaps, double *);

WideFn pick_wide(int L, int KB0)
{
    if (KB0 == 1) {
        switch (L) {
        case 2: return mlp_wide_kernel<2, 1>;
        case 3: return mlp_wide_kernel<3, 1>;
        case 4: return mlp_wide_kernel<4, 1>;
        default: return nullptr;
        }
    }
    if (KB0 == 2) {
        switch (L) {
        case 2: return mlp_wide_kernel<2, 2>;
        case 3: return mlp_wide_kernel<3, 2>;
        case 4: return mlp_wide_kernel<4, 2>;
        default: return nullptr;
        }
    }
    return nullptr;
}

}  // namespace

size_t mlp_wide_smem(int n, int ns) { return wide_layout(n, ns).total; }

bool mlp_wide_supported(int hidden, int layers, int in_pad, int outputs, int n, int ns, int)
{
    return hidden == kHW && in_pad % 8 == 0 && in_pad >= n + 2 && in_pad <= 128 && n + 2 <= kOutW &&
           outputs >= n && ns >= 1 && ns <= kMaxStrikesW && pick_wide(layers, (in_pad + 63) / 64) != nullptr &&
           wide_layout(n, ns).total <= 227 * 1024;
}

int launch_mlp_wide(int layers, int in_pad, int outputs, int grid, cudaStream_t st, const PathArgs &a,
                    const MlpArgs &g, double *acc)
{
    WideFn f = pick_wide(layers, (in_pad + 63) / 64);
    if (!f || layers > kMaxLayersW) return (int)cudaErrorInvalidValue;
    WideMaps maps;
    for (int l = 0; l < layers; ++l) {
        const int din = l == 0 ? in_pad : kHW;
        if (!make_tmap(&maps.w[l], g.wh + g.offW[l], kHW, din, din, kHW)) return (int)cudaErrorInvalidValue;
    }
    if (!make_tmap(&maps.w[layers], g.wh + g.off_wout, outputs, kHW, kHW, kOutW)) return (int)cudaErrorInvalidValue;
    const size_t smem = wide_layout(a.n, a.ns).total;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    f<<<grid, kThreadsW, smem, st>>>(a, g, maps, acc);
    return (int)cudaGetLastError();
}

}  // namespace lll
