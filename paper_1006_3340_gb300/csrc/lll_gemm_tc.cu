// lll_gemm_tc.cu -- the learned compensator's GEMMs on the 5th-generation
// tensor cores: tcgen05.mma with BF16 operands in shared memory and the FP32
// accumulator in tensor memory.
//
// C[M x N] = sum_k A(m, k) B(k, n) over the K range of blockIdx.z, with
//   A(m, k) = A[m lda + k] (TA = 0) or A[k lda + m] (TA = 1),
//   B(k, n) = B[k ldb + n] (TB = 0) or B[n ldb + k] (TB = 1),
// and the epilogues of the training and layer-by-layer inference passes:
//   EPI 0: FP32 C (+ z M N for split-K partials),
//   EPI 1: z = C + bias[n]; Zout = z (FP32, if given); Hout = bf16(SiLU(z)),
//   EPI 2: d = C SiLU'(Zin[m, n]); Zout = d (FP32); Hout = bf16(d),
//   EPI 3: C + bias[n] into C (FP32),
//   EPI 4: C + bias[m] into C (FP32; the vector head's output layer computed
//          transposed, out^T = W_out H^T, so that rates are rows).
// SiLU(z) = z (1 + tanh(z / 2)) / 2 with tanh.approx, the same function as the
// mma.sync kernels and the fused inference kernels.
//
// A CTA computes a 128 x NT tile (NT = 64, 128 or 256): 128 threads, one per
// accumulator row (TMEM lane) in the epilogue, which stages each group of 64
// output columns in shared memory so that global stores are coalesced 16-byte
// chunks.  K advances in blocks of 64.
// Every thread stages part of the A and B blocks into a two-deep ring in the
// 128-byte-swizzled K-major operand layout: K-contiguous sources by cp.async
// (16 bytes, zero-filled past M, N or K), transposed sources (TA = 1, TB = 0)
// by coalesced 2-byte loads gathered into 16-byte chunks.  One thread issues
// the four K = 16 products of a block and commits them to the block's
// mbarrier; the block after next is staged into the same buffer once that
// barrier completes, so staging overlaps the products.  Waits are bounded: a
// wait that runs out sets the launch's error word, the CTA drains its
// products through a final commit and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/lll.h"
#include "lll_internal.h"
#include "lll_mlp.h"
#include "lll_tc.cuh"

namespace lll {
namespace {

constexpr int kM = 128;                      // rows per CTA tile (TMEM lanes)
constexpr int kWsMinRows = 8192;             // streamed rows from which the weight-stationary kernel is used
constexpr int kThreadsG = 128;

struct GemmArgs {
    const __nv_bfloat16 *A;
    const __nv_bfloat16 *B;
    int lda, ldb, M, N, K, k_chunk;
    float *C;
    const float *bias, *Zin;
    float *Zout;
    __nv_bfloat16 *Hout;
    int vecA, vecB; // 1: the K-contiguous operand is 16-byte aligned (cp.async path)
    int *err;
};

using namespace tc;

// D FP32, A and B BF16, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc(int n) { return idesc_m128(n); }

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Bounded wait for phase parity `par` of barrier b; false when it gave up
// (then the launch's error word is set).  Only thread 0 of a CTA waits; the
// CTA learns the outcome through __syncthreads_or, so every thread takes the
// same branch.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t par, int *err)
{
    const uint32_t a = saddr(b);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(a), "r"(par)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitBudget) {
            atomicOr(err, 1);
            return false;
        }
    }
}

// 16 accumulator columns of this thread's TMEM lane, waited for.
__device__ __forceinline__ void tmem_ld16_wait(uint32_t ta, uint32_t (&r)[16])
{
    tmem_ld16(ta, r);
    tmem_wait(r);
}

__device__ __forceinline__ float silu(float z) { return 0.5f * z * (1.0f + tanh_approx(0.5f * z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 0.5f * (1.0f + tanh_approx(0.5f * z));
    return s * (1.0f + z * (1.0f - s));
}

// Stage rows [r0, r0 + R) of one operand's 64-wide K block starting at k0
// (k < kend valid) into the swizzled block at `dst`.  TRANS = 0: element
// (row, k) at P[row ld + k]; TRANS = 1: at P[k ld + row].  rows_valid: rows
// beyond it are zero.
template <int R, int TRANS>
__device__ __forceinline__ void stage_operand(uint32_t dst, const __nv_bfloat16 *P, int ld, int r0, int rows_valid,
                                              int k0, int kend, bool vec, int tid = threadIdx.x,
                                              int nthr = kThreadsG)
{
    if (!TRANS) {
        // chunk e = (row, c8); consecutive threads take consecutive chunks of a row
        for (int e = tid; e < R * 8; e += nthr) {
            const int r = e >> 3, c8 = e & 7;
            const int k = k0 + c8 * 8;
            const int row = r0 + r;
            int valid = (row < rows_valid) ? min(max(kend - k, 0), 8) : 0;
            const uint32_t d = dst + swz(r, c8);
            if (vec) {
                const __nv_bfloat16 *src = valid > 0 ? P + (size_t)row * ld + k : P;
                cp_async16_zfill(d, src, valid * 2);
            } else {
                uint32_t w[4] = {0, 0, 0, 0};
                for (int j = 0; j < valid; ++j) {
                    const uint32_t v = __bfloat16_as_ushort(P[(size_t)row * ld + k + j]);
                    w[j >> 1] |= v << ((j & 1) * 16);
                }
                asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(d), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                             "r"(w[3])
                             : "memory");
            }
        }
    } else {
        // chunk e = (c8, row): consecutive threads take consecutive rows, so each
        // of the 8 loads of a chunk is coalesced across the warp
        for (int e = tid; e < R * 8; e += nthr) {
            const int c8 = e / R, r = e % R;
            const int row = r0 + r;
            uint32_t w[4] = {0, 0, 0, 0};
            if (row < rows_valid) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + c8 * 8 + j;
                    if (k < kend) {
                        const uint32_t v = __bfloat16_as_ushort(P[(size_t)k * ld + row]);
                        w[j >> 1] |= v << ((j & 1) * 16);
                    }
                }
            }
            asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(dst + swz(r, c8)), "r"(w[0]), "r"(w[1]),
                         "r"(w[2]), "r"(w[3])
                         : "memory");
        }
    }
}

template <int TA, int TB, int EPI, int NT>
__global__ void __launch_bounds__(kThreadsG) gemm_tc(const GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_g[];
    constexpr uint32_t kAB = kM * 128, kBB = NT * 128, kStage = kAB + kBB;
    __shared__ uint64_t done[2], fin;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kM, n0 = blockIdx.x * NT;
    const int kbeg = blockIdx.z * g.k_chunk, kend = min(g.K, kbeg + g.k_chunk);
    const int nkb = kend > kbeg ? (kend - kbeg + 63) / 64 : 0;
    // the ring starts at a 1024-byte boundary (the swizzle atom)
    const uint32_t base = (saddr(smem_g) + 1023u) & ~1023u;
    if (tid == 0) {
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        mbar_init(&fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tslot)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t id = idesc(NT);

    auto stage = [&](int buf, int kb) {
        const uint32_t sa = base + buf * kStage, sb = sa + kAB;
        const int k0 = kbeg + kb * 64;
        stage_operand<kM, TA>(sa, g.A, g.lda, m0, g.M, k0, kend, g.vecA != 0);
        stage_operand<NT, TB ? 0 : 1>(sb, g.B, g.ldb, n0, g.N, k0, kend, g.vecB != 0);
    };

    if (nkb > 0) stage(0, 0);
    cp_commit();
    bool bad = false;
    for (int i = 0; i < nkb; ++i) {
        const int s = i & 1;
        if (i + 1 < nkb) {
            // buffer s ^ 1 was read by the products of block i - 1
            bool gave_up = false;
            if (i >= 1 && tid == 0) gave_up = !mbar_wait_bounded(&done[s ^ 1], ((i - 1) >> 1) & 1, g.err);
            if (__syncthreads_or(gave_up)) {
                bad = true;
                break;
            }
            stage(s ^ 1, i + 1);
            cp_commit();
            cp_wait_1();
        } else {
            cp_wait_0();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_after();
            const uint32_t sa = base + s * kStage, sb = sa + kAB;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_ss(tmem, sdesc(sa + ks * 32), sdesc(sb + ks * 32), id, (i > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&done[s]);
        }
    }
    cp_wait_0();
    // every product of this CTA has completed once the final commit arrives
    bool gave_up = false;
    if (tid == 0) {
        if (nkb > 0) mma_commit(&fin);
        else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&fin)) : "memory");
        gave_up = !mbar_wait_bounded(&fin, 0, g.err);
    }
    bad = __syncthreads_or(gave_up || bad);
    tc_after();

    // Epilogue in groups of 64 columns: each thread reads its accumulator row
    // (TMEM lane) and writes the group's outputs into shared memory (the
    // operand ring is free now), then the CTA writes them to global memory
    // in coalesced 16-byte chunks.
    const int rloc = warp * 32 + lane;
    if (!bad) {
        constexpr int CG = 64;
        constexpr int FP = CG + 4;                           // FP32 staging pitch (floats)
        constexpr int HP = CG + 8;                           // BF16 staging pitch (elements)
        float *sf = reinterpret_cast<float *>(smem_g + (base - saddr(smem_g)));        // [128][FP]
        __nv_bfloat16 *sh = reinterpret_cast<__nv_bfloat16 *>(sf + kM * FP);         // [128][HP]
        const bool vecf = (g.N % 4) == 0, vech = (g.N % 8) == 0;
        float *fout = EPI == 0 ? g.C + (size_t)blockIdx.z * g.M * g.N : ((EPI == 3 || EPI == 4) ? g.C : g.Zout);
        for (int cg0 = 0; cg0 < NT; cg0 += CG) {
            if (cg0 >= g.N - n0) break; // uniform: no valid column left in this tile
#pragma unroll
            for (int c16 = 0; c16 < CG; c16 += 16) {
                uint32_t r[16];
                if (nkb > 0) {
                    tmem_ld16_wait(tmem + ((uint32_t)(warp * 32) << 16) + cg0 + c16, r);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) r[j] = 0u;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int cl = c16 + j, gn = n0 + cg0 + cl;
                    const float v = __uint_as_float(r[j]);
                    float f = v;
                    if (EPI == 1 || EPI == 3) f = v + (gn < g.N ? g.bias[gn] : 0.0f);
                    if (EPI == 4) f = v + (m0 + rloc < g.M ? g.bias[m0 + rloc] : 0.0f);
                    // epilogue 2 applies SiLU'(Zin) in the copy-out below, where Zin is
                    // read along rows (coalesced)
                    sf[rloc * FP + cl] = f;
                    if (EPI == 1) sh[rloc * HP + cl] = __float2bfloat16(silu(f));
                }
            }
            __syncthreads();
            const int rows = min(kM, g.M - m0), cols = min(CG, g.N - n0 - cg0);
            if (EPI == 2) {
                // d = C SiLU'(Zin): FP32 to Zout and BF16 to Hout along rows
                // (consecutive threads, consecutive 4-column chunks); four chunks per
                // thread are loaded before any is used, so the loads overlap
                if (vecf && cols == CG) {
                    constexpr int CH = CG / 4;
                    for (int q0 = tid; q0 < rows * CH; q0 += 4 * kThreadsG) {
                        float4 z[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = q0 + u * kThreadsG;
                            if (q < rows * CH)
                                z[u] = __ldg(reinterpret_cast<const float4 *>(
                                    g.Zin + (size_t)(m0 + q / CH) * g.N + n0 + cg0 + (q % CH) * 4));
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = q0 + u * kThreadsG;
                            if (q >= rows * CH) break;
                            const int rr = q / CH, cc = (q % CH) * 4;
                            const size_t o = (size_t)(m0 + rr) * g.N + n0 + cg0 + cc;
                            const float4 a = *reinterpret_cast<const float4 *>(sf + rr * FP + cc);
                            const float4 d = make_float4(a.x * silu_grad(z[u].x), a.y * silu_grad(z[u].y),
                                                         a.z * silu_grad(z[u].z), a.w * silu_grad(z[u].w));
                            *reinterpret_cast<float4 *>(g.Zout + o) = d;
                            const __nv_bfloat162 h0 = __floats2bfloat162_rn(d.x, d.y), h1 = __floats2bfloat162_rn(d.z, d.w);
                            uint2 hw;
                            hw.x = *reinterpret_cast<const uint32_t *>(&h0);
                            hw.y = *reinterpret_cast<const uint32_t *>(&h1);
                            *reinterpret_cast<uint2 *>(g.Hout + o) = hw;
                        }
                    }
                } else {
                    for (int q = tid; q < rows * CG; q += kThreadsG) {
                        const int rr = q / CG, cc = q % CG;
                        if (cc >= cols) continue;
                        const size_t o = (size_t)(m0 + rr) * g.N + n0 + cg0 + cc;
                        const float d = sf[rr * FP + cc] * silu_grad(g.Zin[o]);
                        g.Zout[o] = d;
                        g.Hout[o] = __float2bfloat16(d);
                    }
                }
                __syncthreads();
                continue;
            }
            const bool want_f = EPI != 1 || g.Zout != nullptr;
            if (want_f) {
                if (vecf) {
                    for (int q = tid; q < rows * (CG / 4); q += kThreadsG) {
                        const int rr = q / (CG / 4), cc = (q % (CG / 4)) * 4;
                        if (cc >= cols) continue;
                        float *dst = fout + (size_t)(m0 + rr) * g.N + n0 + cg0 + cc;
                        *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(sf + rr * FP + cc);
                    }
                } else {
                    for (int q = tid; q < rows * CG; q += kThreadsG) {
                        const int rr = q / CG, cc = q % CG;
                        if (cc < cols) fout[(size_t)(m0 + rr) * g.N + n0 + cg0 + cc] = sf[rr * FP + cc];
                    }
                }
            }
            if (EPI == 1) {
                if (vech) {
                    for (int q = tid; q < rows * (CG / 8); q += kThreadsG) {
                        const int rr = q / (CG / 8), cc = (q % (CG / 8)) * 8;
                        if (cc >= cols) continue;
                        __nv_bfloat16 *dst = g.Hout + (size_t)(m0 + rr) * g.N + n0 + cg0 + cc;
                        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(sh + rr * HP + cc);
                    }
                } else {
                    for (int q = tid; q < rows * CG; q += kThreadsG) {
                        const int rr = q / CG, cc = q % CG;
                        if (cc < cols) g.Hout[(size_t)(m0 + rr) * g.N + n0 + cg0 + cc] = sh[rr * HP + cc];
                    }
                }
            }
            __syncthreads();
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

// ---------------------------------------------------------------------------
// Weight-stationary persistent variant for the network's forward products
// (K <= 256, many rows): the stationary operand (a layer's weights, at most
// 256 x 256 BF16 = 128 KB) is staged into shared memory once per CTA and the
// CTA loops over tiles of the streamed operand (the activation rows).
// Warp roles: warps 0-7 epilogue (warp w reads TMEM lanes 32 (w mod 4) ..
// + 31 and column half w div 4; each stages its 32 x 32 blocks in its own
// shared-memory slot and writes them out in coalesced row segments), warp 8
// lane 0 the producer (one TMA box per streamed 64-wide K block,
// cp.async.bulk.tensor with 128-byte swizzle into a ring, completion counted
// in bytes on the stage's mbarrier), warp 9 lane 0 issues the products into
// one of two TMEM accumulators, so the epilogue of one tile runs under the
// products of the next.
//   SA = 0: B stationary (W [N x K], N <= NT), A streamed in 128-row tiles;
//           EPI 1 (a hidden layer: bias[n] + SiLU -> BF16 H, FP32 Z if given).
//   SA = 1: A stationary (W_out [M x K], M <= 128), B streamed in 256-row
//           tiles of activation rows; EPI 4 (out^T = W_out H^T + bias[m]).
// Every wait is bounded: on timeout the CTA's abort flag and the launch's
// error word are set, every role leaves its loop, the MMA lane drains its
// products through a final commit and the tensor memory is freed.
constexpr int kWsEpiWarps = 8;                         // 4 TMEM lane quadrants x 2 column halves
constexpr int kWsThreads = (kWsEpiWarps + 2) * 32;      // + producer warp + MMA warp
constexpr int kWsFP = 36;                               // staging pitch (floats) of a warp's 32 x 32 block
constexpr uint32_t kWsStageBytes = 32 * kWsFP * 4;      // per epilogue warp

template <int SA>
struct WsShape {
    static constexpr int TR = SA ? 256 : 128;  // rows of a streamed tile
    static constexpr uint32_t KBLK = TR * 128; // bytes of one streamed 64-wide K block
    static constexpr int STG = SA ? 2 : 3;     // ring stages (64 / 48 KB)
};

template <int SA, int EPI, int NT>
__global__ void __launch_bounds__(kWsThreads, 1) gemm_ws(const GemmArgs g, const __grid_constant__ CUtensorMap tmap)
{
    using S = WsShape<SA>;
    constexpr int SR = SA ? kM : NT;           // rows of the stationary operand
    constexpr uint32_t SBLK = SR * 128;        // bytes of one stationary K block
    constexpr int MN = SA ? S::TR : NT;        // product N (accumulator columns)
    extern __shared__ __align__(1024) unsigned char smem_w[];
    __shared__ uint64_t full[S::STG], empty[S::STG], accf[2], acce[2], fin;
    __shared__ uint32_t tslot;
    __shared__ int abort_w;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KB = (g.K + 63) / 64; // <= 4
    const uint32_t base = (saddr(smem_w) + 1023u) & ~1023u;
    const uint32_t sst = base, sring = base + 4 * SBLK, sstage = sring + S::STG * S::KBLK;
    const int ntiles = SA ? (g.N + S::TR - 1) / S::TR : (g.M + kM - 1) / kM;
    volatile int *abort = &abort_w;
    if (tid == 0) {
        for (int i = 0; i < S::STG; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], kWsEpiWarps);
        }
        mbar_init(&fin, 1);
        abort_w = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tslot)),
                     "r"(2 * MN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the stationary operand, every K block, by the whole CTA
    for (int kb = 0; kb < KB; ++kb) {
        if (SA) stage_operand<SR, 0>(sst + kb * SBLK, g.A, g.lda, 0, g.M, kb * 64, g.K, g.vecA != 0, tid, kWsThreads);
        else stage_operand<SR, 0>(sst + kb * SBLK, g.B, g.ldb, 0, g.N, kb * 64, g.K, g.vecB != 0, tid, kWsThreads);
    }
    cp_commit();
    cp_wait_0();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tslot;

    if (warp == kWsEpiWarps) {
        // ---------------- producer: one TMA box per streamed K block ----------------
        if (lane == 0) {
            const uint64_t tm = reinterpret_cast<uint64_t>(&tmap);
            asm volatile("prefetch.tensormap [%0];" ::"l"(tm) : "memory");
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % S::STG, u = it / S::STG;
                    if (u >= 1 && !(ok = mbar_wait(&empty[s], (u - 1) & 1, abort, g.err))) break;
                    const uint32_t bar = saddr(&full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                                 "r"(S::KBLK)
                                 : "memory");
                    // box {64 K elements, TR rows} at (k = 64 kb, row = TR t); rows past the
                    // tensor are filled with zeros
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(sring + s * S::KBLK),
                                 "l"(tm), "r"(kb * 64), "r"(t * S::TR), "r"(bar)
                                 : "memory");
                }
            }
        }
        __syncwarp();
    } else if (warp == kWsEpiWarps + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MN >> 3) << 17) |
                                    ((uint32_t)(kM >> 4) << 24);
            int it = 0, j = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++j) {
                const int b = j & 1, v = j >> 1;
                if (v >= 1 && !(ok = mbar_wait(&acce[b], (v - 1) & 1, abort, g.err))) break;
                tc_after();
                const uint32_t d = tmem + b * MN;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % S::STG, u = it / S::STG;
                    if (!(ok = mbar_wait(&full[s], u & 1, abort, g.err))) break;
                    tc_after();
                    const uint32_t rb = sring + s * S::KBLK, sb = sst + kb * SBLK;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = sdesc((SA ? sb : rb) + ks * 32), bd = sdesc((SA ? rb : sb) + ks * 32);
                        mma_ss(d, ad, bd, id, (kb > 0 || ks > 0) ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&accf[b]);
            }
            // every product issued by this lane has completed once this arrives
            mma_commit(&fin);
            mbar_wait(&fin, 0, abort, g.err);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warp w = lane quadrant w % 4, column half w / 4 ----------------
        const int q = warp & 3, half = warp >> 2;
        unsigned char *slot = smem_w + (sstage - saddr(smem_w)) + warp * kWsStageBytes;
        float *sf = reinterpret_cast<float *>(slot);                 // [32][kWsFP]
        __nv_bfloat16 *sh = reinterpret_cast<__nv_bfloat16 *>(slot); // [32][2 kWsFP]
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int b = j & 1, v = j >> 1;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&accf[b], v & 1, abort, g.err);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc_after();
            const int r0 = (SA ? 0 : t * kM) + q * 32, c0 = SA ? t * S::TR : 0;
            const int rows = min(32, g.M - r0), cols = min(MN, g.N - c0);
            const int m = r0 + lane; // this thread's accumulator row
            for (int cg = half * (MN / 2); cg < (half + 1) * (MN / 2) && cg < cols; cg += 32) {
                uint32_t r[2][16];
                tmem_ld16_wait(tmem + ((uint32_t)(q * 32) << 16) + b * MN + cg, r[0]);
                tmem_ld16_wait(tmem + ((uint32_t)(q * 32) << 16) + b * MN + cg + 16, r[1]);
                float f[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float acc = __uint_as_float(r[c >> 4][c & 15]);
                    const int n = c0 + cg + c;
                    f[c] = acc;
                    if (EPI == 1) f[c] = acc + (n < g.N ? __ldg(g.bias + n) : 0.0f);
                    if (EPI == 4) f[c] = acc + (m < g.M ? __ldg(g.bias + m) : 0.0f);
                }
                const int cc_n = min(32, cols - cg);
                // FP32 values (the output of epilogue 4, or the pre-activations): 16-byte
                // stores at pitch 36 floats are conflict-free; then each row's 128 bytes
                // go out as 8 chunks, 4 rows per warp instruction
                if (EPI == 4 || g.Zout != nullptr) {
                    float *fout = EPI == 4 ? g.C : g.Zout;
#pragma unroll
                    for (int c = 0; c < 32; c += 4)
                        *reinterpret_cast<float4 *>(sf + lane * kWsFP + c) = make_float4(f[c], f[c + 1], f[c + 2], f[c + 3]);
                    __syncwarp();
                    for (int e = lane; e < rows * 8; e += 32) {
                        const int rr = e >> 3, cc = (e & 7) * 4;
                        float *dst = fout + (size_t)(r0 + rr) * g.N + c0 + cg + cc;
                        if ((g.N % 4) == 0 && cc + 4 <= cc_n) {
                            *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(sf + rr * kWsFP + cc);
                        } else {
                            for (int x = 0; x < 4 && cc + x < cc_n; ++x) dst[x] = sf[rr * kWsFP + cc + x];
                        }
                    }
                    __syncwarp();
                }
                if (EPI == 1) {
                    // BF16 SiLU activations: 4 chunks of 8 per row (pitch 72 elements)
#pragma unroll
                    for (int c = 0; c < 32; c += 8) {
                        uint4 w;
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(silu(f[c]), silu(f[c + 1]));
                        __nv_bfloat162 h1 = __floats2bfloat162_rn(silu(f[c + 2]), silu(f[c + 3]));
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(silu(f[c + 4]), silu(f[c + 5]));
                        __nv_bfloat162 h3 = __floats2bfloat162_rn(silu(f[c + 6]), silu(f[c + 7]));
                        w.x = *reinterpret_cast<uint32_t *>(&h0);
                        w.y = *reinterpret_cast<uint32_t *>(&h1);
                        w.z = *reinterpret_cast<uint32_t *>(&h2);
                        w.w = *reinterpret_cast<uint32_t *>(&h3);
                        *reinterpret_cast<uint4 *>(sh + lane * (2 * kWsFP) + c) = w;
                    }
                    __syncwarp();
                    for (int e = lane; e < rows * 4; e += 32) {
                        const int rr = e >> 2, cc = (e & 3) * 8;
                        __nv_bfloat16 *dst = g.Hout + (size_t)(r0 + rr) * g.N + c0 + cg + cc;
                        if ((g.N % 8) == 0 && cc + 8 <= cc_n) {
                            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(sh + rr * (2 * kWsFP) + cc);
                        } else {
                            for (int x = 0; x < 8 && cc + x < cc_n; ++x) dst[x] = sh[rr * (2 * kWsFP) + cc + x];
                        }
                    }
                    __syncwarp();
                }
            }
            // this warp's share of the accumulator has been read
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * MN));
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

}  // namespace

// Tensor map of a row-major BF16 matrix [rows x K] (leading dimension ld
// elements, a multiple of 8) read in boxes of {64, box_rows} with the
// 128-byte swizzle of the K-major operand layout.
bool make_tmap(CUtensorMap *tm, const void *base, int rows, int K, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// Returns cudaErrorNotSupported (no launch) when the tensor map cannot be made;
// the caller then uses the general kernel.
template <int SA, int EPI, int NT>
int launch_ws(cudaStream_t st, const GemmArgs &g, int sms)
{
    using S = WsShape<SA>;
    constexpr int SR = SA ? kM : NT;
    CUtensorMap tm;
    if (!(SA ? make_tmap(&tm, g.B, g.N, g.K, g.ldb, S::TR) : make_tmap(&tm, g.A, g.M, g.K, g.lda, S::TR)))
        return (int)cudaErrorNotSupported;
    const size_t smem = 4 * (size_t)SR * 128 + (size_t)S::STG * S::KBLK + kWsEpiWarps * (size_t)kWsStageBytes + 1024;
    auto kern = gemm_ws<SA, EPI, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int ntiles = SA ? (g.N + S::TR - 1) / S::TR : (g.M + kM - 1) / kM;
    kern<<<ntiles < sms ? ntiles : sms, kWsThreads, smem, st>>>(g, tm);
    return (int)cudaGetLastError();
}

template <int TA, int TB, int EPI>
int launch_nt(int NT, dim3 grid, cudaStream_t st, const GemmArgs &g)
{
    auto run = [&](auto kern, int nt) -> int {
        // the operand ring, or the epilogue's staging of 64 columns (FP32 and
        // BF16 copies) if larger, plus the alignment slack
        const size_t ring = 2 * (size_t)(kM * 128 + nt * 128);
        const size_t epi_stage = (size_t)kM * (64 + 4) * 4 + (size_t)kM * (64 + 8) * 2;
        const size_t smem = (ring > epi_stage ? ring : epi_stage) + 1024;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        kern<<<grid, kThreadsG, smem, st>>>(g);
        return (int)cudaGetLastError();
    };
    if (NT == 64) return run(gemm_tc<TA, TB, EPI, 64>, 64);
    if (NT == 128) return run(gemm_tc<TA, TB, EPI, 128>, 128);
    return run(gemm_tc<TA, TB, EPI, 256>, 256);
}

// Error word of the launches on this device (bounded waits that gave up).
__device__ int g_gemm_err;

int g_gemm_kind = LLL_GEMM_TC; // process-wide choice (lll_set_gemm_kernel)

}  // namespace

int mlp_gemm(int ta, int tb, int epi, const void *A, int lda, const void *B, int ldb, int M, int N, int K,
             int splits, float *C, const float *bias, const float *Zin, float *Zout, void *Hout, cudaStream_t st)
{
    if (g_gemm_kind == LLL_GEMM_MMA_SYNC)
        return mlp_gemm_mma(ta, tb, epi, A, lda, B, ldb, M, N, K, splits, C, bias, Zin, Zout, Hout, st);
    int *err = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_gemm_err);
    if (e != cudaSuccess) return (int)e;
    return mlp_gemm_tc(ta, tb, epi, A, lda, B, ldb, M, N, K, splits, C, bias, Zin, Zout, Hout, err, st);
}

int mlp_gemm_kind() { return g_gemm_kind; }

int mlp_splits_used(int K, int splits)
{
    return g_gemm_kind == LLL_GEMM_MMA_SYNC ? mlp_splits_used_mma(K, splits) : mlp_splits_used_tc(K, splits);
}

int mlp_gemm_take_error(int *word, cudaStream_t st)
{
    int *err = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_gemm_err);
    if (e == cudaSuccess) e = cudaMemcpyAsync(word, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return (int)e;
}

// The same contract as mlp_gemm's mma.sync kernel (lll_mlp.cu).
int mlp_gemm_tc(int ta, int tb, int epi, const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                int splits, float *C, const float *bias, const float *Zin, float *Zout, void *Hout, int *err,
                cudaStream_t st)
{
    if (splits < 1) splits = 1;
    int k_chunk = (K + splits - 1) / splits;
    k_chunk = ((k_chunk + 63) / 64) * 64;
    splits = (K + k_chunk - 1) / k_chunk;
    const int NT = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
    dim3 grid((N + NT - 1) / NT, (M + kM - 1) / kM, splits);
    GemmArgs g{};
    g.A = static_cast<const __nv_bfloat16 *>(A);
    g.B = static_cast<const __nv_bfloat16 *>(B);
    g.lda = lda; g.ldb = ldb; g.M = M; g.N = N; g.K = K; g.k_chunk = k_chunk;
    g.C = C; g.bias = bias; g.Zin = Zin; g.Zout = Zout; g.Hout = static_cast<__nv_bfloat16 *>(Hout);
    // cp.async needs 16-byte aligned rows: the base and the leading dimension
    g.vecA = (!ta && ((uintptr_t)A % 16) == 0 && lda % 8 == 0) ? 1 : 0;
    g.vecB = (tb && ((uintptr_t)B % 16) == 0 && ldb % 8 == 0) ? 1 : 0;
    g.err = err;
    // tall-skinny forward products (K a multiple of 64, at most 256): the
    // weight-stationary persistent kernel, streaming the activations by TMA
    if (ta == 0 && tb == 1 && K <= 256 && K % 64 == 0 && splits == 1) {
        int dev = 0, sms = 0;
        int rc = (int)cudaErrorNotSupported;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
            if (epi == 1 && N <= 256 && M >= kWsMinRows && g.vecA) {
                if (N <= 64) rc = launch_ws<0, 1, 64>(st, g, sms);
                else if (N <= 128) rc = launch_ws<0, 1, 128>(st, g, sms);
                else rc = launch_ws<0, 1, 256>(st, g, sms);
            } else if (epi == 4 && M <= kM && N >= kWsMinRows && g.vecB) {
                rc = launch_ws<1, 4, 256>(st, g, sms);
            }
        }
        if (rc != (int)cudaErrorNotSupported) return rc;
    }
    if (epi == 0 && ta == 0 && tb == 0) return launch_nt<0, 0, 0>(NT, grid, st, g);
    if (epi == 0 && ta == 1 && tb == 0) return launch_nt<1, 0, 0>(NT, grid, st, g);
    if (epi == 0 && ta == 0 && tb == 1) return launch_nt<0, 1, 0>(NT, grid, st, g);
    if (epi == 1 && ta == 0 && tb == 1) return launch_nt<0, 1, 1>(NT, grid, st, g);
    if (epi == 2 && ta == 0 && tb == 0) return launch_nt<0, 0, 2>(NT, grid, st, g);
    if (epi == 2 && ta == 0 && tb == 1) return launch_nt<0, 1, 2>(NT, grid, st, g);
    if (epi == 3 && ta == 0 && tb == 1) return launch_nt<0, 1, 3>(NT, grid, st, g);
    if (epi == 4 && ta == 0 && tb == 1) return launch_nt<0, 1, 4>(NT, grid, st, g);
    return (int)cudaErrorInvalidValue;
}

int mlp_splits_used_tc(int K, int splits)
{
    if (splits < 1) splits = 1;
    int k_chunk = (K + splits - 1) / splits;
    k_chunk = ((k_chunk + 63) / 64) * 64;
    return (K + k_chunk - 1) / k_chunk;
}

}  // namespace lll

extern "C" int lll_set_gemm_kernel(int kind)
{
    if (kind != LLL_GEMM_TC && kind != LLL_GEMM_MMA_SYNC)
        return lll::record_error(nullptr, LLL_EINVAL, "kind must be LLL_GEMM_TC or LLL_GEMM_MMA_SYNC");
    lll::g_gemm_kind = kind;
    return LLL_OK;
}

// One product of the current GEMM kernel on host buffers (see lll.h).
extern "C" int lll_gemm_bf16(int ta, int tb, int epi, const uint16_t *A, int lda, const uint16_t *B, int ldb, int M,
                             int N, int K, int splits, const float *bias, const float *Zin, float *C, uint16_t *H)
{
    using namespace lll;
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || splits < 1 || lda < 1 || ldb < 1)
        return record_error(nullptr, LLL_EINVAL, "null buffer or non-positive size");
    if ((epi == 1 && (!bias || !H)) || (epi == 2 && (!Zin || !H)) || (epi >= 3 && !bias) || epi < 0 || epi > 4)
        return record_error(nullptr, LLL_EINVAL, "epilogue 1 needs bias and H, 2 Zin and H, 3 and 4 bias");
    if ((epi == 0 && tb == 1 && ta == 1) || ((epi == 1 || epi >= 3) && (ta || !tb)) || (epi == 2 && ta) ||
        (epi == 2 && tb && g_gemm_kind != LLL_GEMM_TC))
        return record_error(nullptr, LLL_EUNSUPPORTED, "operand layout not used with this epilogue");
    if (epi >= 3 && g_gemm_kind != LLL_GEMM_TC)
        return record_error(nullptr, LLL_EUNSUPPORTED, "epilogues 3 and 4 are tcgen05 only");
    const size_t na = (size_t)(ta ? K : M) * lda, nb = (size_t)(tb ? N : K) * ldb, mn = (size_t)M * N;
    const int used = epi == 0 ? mlp_splits_used(K, splits) : 1;
    void *dA = nullptr, *dB = nullptr, *dH = nullptr;
    float *dC = nullptr, *dbias = nullptr, *dZin = nullptr;
    cudaError_t e = cudaMalloc(&dA, 2 * na);
    if (e == cudaSuccess) e = cudaMalloc(&dB, 2 * nb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dC, 4 * mn * used);
    const size_t nbias = epi == 4 ? (size_t)M : (size_t)N;
    if (e == cudaSuccess && (epi == 1 || epi == 2)) e = cudaMalloc(&dH, 2 * mn);
    if (e == cudaSuccess && (epi == 1 || epi >= 3)) e = cudaMalloc((void **)&dbias, 4 * nbias);
    if (e == cudaSuccess && epi == 2) e = cudaMalloc((void **)&dZin, 4 * mn);
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, 2 * na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, 2 * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && (epi == 1 || epi >= 3)) e = cudaMemcpy(dbias, bias, 4 * nbias, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && epi == 2) e = cudaMemcpy(dZin, Zin, 4 * mn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = (cudaError_t)mlp_gemm(ta, tb, epi, dA, lda, dB, ldb, M, N, K, splits,
                                  (epi == 0 || epi >= 3) ? dC : nullptr, dbias, dZin,
                                  (epi == 1 || epi == 2) ? dC : nullptr, dH, nullptr);
    std::vector<float> part;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && epi == 0) {
        part.resize(mn * used);
        e = cudaMemcpy(part.data(), dC, 4 * mn * used, cudaMemcpyDeviceToHost);
        for (size_t o = 0; o < mn && e == cudaSuccess; ++o) {
            float acc = 0.0f;
            for (int z = 0; z < used; ++z) acc += part[(size_t)z * mn + o];
            C[o] = acc;
        }
    } else if (e == cudaSuccess) {
        e = cudaMemcpy(C, dC, 4 * mn, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && dH) e = cudaMemcpy(H, dH, 2 * mn, cudaMemcpyDeviceToHost);
    }
    int word = 0;
    if (e == cudaSuccess && g_gemm_kind == LLL_GEMM_TC) e = (cudaError_t)mlp_gemm_take_error(&word, nullptr);
    cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(dH); cudaFree(dbias); cudaFree(dZin);
    if (e != cudaSuccess) return record_error(nullptr, LLL_ECUDA, cudaGetErrorString(e));
    if (word) return record_error(nullptr, LLL_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up");
    return LLL_OK;
}
