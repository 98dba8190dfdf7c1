// lll_mlp_layered.cu -- the learned-compensator scheme (LLL_MLP) for networks
// the fused kernels cannot hold (hidden width 256, wide inputs, the vector
// head): the network runs layer by layer over all rows of a step with the
// training GEMMs, between two small kernels of this file.  A row is one
// (path, live rate), or one path for the vector head, whose output layer gives
// every rate's compensator at once.
//
// Per Euler step k of Eq. (log-LIB-SDE-2), for a chunk of paths:
//  feat_kernel   one BF16 feature row x_i = (t s_t, i s_i, lambda_i s_lam,
//                u_0 .. u_{N-1}) per (path, live rate), row = p * live + (i - imin);
//  (network)     f(x) for every row, FP32 (lll_mlp.cu);
//  euler_kernel  one thread per path: draws Delta H_k, applies
//                A_i = C_i + s_y f(x_i) (Eq. (LIBOR-drift-PT) with the learned
//                compensator), records the caplet payoffs of Eq. (caplet) at
//                T_m into per-block FP64 Kahan accumulators.
// Blocks own fixed path slots across chunks and steps, so the final
// block-ordered sum is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lll_device.cuh"
#include "lll_internal.h"
#include "lll_mlp.h"

namespace lll {
namespace {

constexpr int kT = 256; // threads per block of both kernels

// Vector head: one row per path, (t s_t, u_0 .. u_{N-1}), written as
// 16-byte chunks.  The path state is [rate][path]: a block stages the state of
// its kFV paths in shared memory (coalesced loads along paths), then writes
// the BF16 rows chunk by chunk (coalesced stores along a row).
constexpr int kFV = 32; // paths per block of feat_vec_kernel

__global__ void __launch_bounds__(kT) feat_vec_kernel(const PathArgs a, MlpScales sc, int k, int Pc,
                                                      const float *state, __nv_bfloat16 *X, int in_pad)
{
    extern __shared__ float fst[]; // [n][kFV + 1]
    const int n = a.n, p0 = blockIdx.x * kFV;
    for (int e = threadIdx.x; e < n * kFV; e += kT) {
        const int m = e / kFV, q = e % kFV;
        fst[m * (kFV + 1) + q] = p0 + q < Pc ? state[(size_t)m * Pc + p0 + q] * sc.u_scale : 0.0f;
    }
    __syncthreads();
    const float t = (float)k * a.h * sc.t_scale;
    const int chunks = in_pad / 8;
    for (int e = threadIdx.x; e < kFV * chunks; e += kT) {
        const int q = e / chunks, ch = e % chunks;
        if (p0 + q >= Pc) continue;
        // columns: 0 t, 1 u_0 = 0, 1 + m  u_m (m = 1..n), then zeros
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = ch * 8 + j, m = c - 1;
            v[j] = c == 0 ? t : ((m >= 1 && m <= n) ? fst[(m - 1) * (kFV + 1) + q] : 0.0f);
        }
        uint4 w;
        __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]), b1 = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[4], v[5]), b3 = __floats2bfloat162_rn(v[6], v[7]);
        w.x = *reinterpret_cast<uint32_t *>(&b0);
        w.y = *reinterpret_cast<uint32_t *>(&b1);
        w.z = *reinterpret_cast<uint32_t *>(&b2);
        w.w = *reinterpret_cast<uint32_t *>(&b3);
        *reinterpret_cast<uint4 *>(X + (size_t)(p0 + q) * in_pad + ch * 8) = w;
    }
}

__global__ void feat_kernel(const PathArgs a, MlpScales sc, int k, int Pc, const float *state,
                            __nv_bfloat16 *X, int in_pad)
{
    const int n = a.n, imin = k / a.s + 1, live = n - imin + 1;
    const size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (size_t)Pc * live) return;
    const int p = (int)(row / live), i = imin + (int)(row % live);
    const float lam = a.row[(size_t)k * n + (i - 1)].x;
    __nv_bfloat162 *x = reinterpret_cast<__nv_bfloat162 *>(X + row * in_pad);
    // columns: 0 t, 1 i, 2 lambda_i, 3 u_0 = 0, 3 + m  u_m (m = 1..n), then zeros
    x[0] = __floats2bfloat162_rn((float)k * a.h * sc.t_scale, (float)i * sc.i_scale);
    x[1] = __floats2bfloat162_rn(lam * sc.lam_scale, 0.0f);
    for (int c = 4; c < in_pad; c += 2) {
        const int m0 = c - 3, m1 = c - 2;
        const float v0 = m0 <= n ? state[(size_t)(m0 - 1) * Pc + p] * sc.u_scale : 0.0f;
        const float v1 = m1 <= n ? state[(size_t)(m1 - 1) * Pc + p] * sc.u_scale : 0.0f;
        x[c / 2] = __floats2bfloat162_rn(v0, v1);
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void kahan_add(double *s, double *c, double x)
{
    const double y = x - *c;
    const double t = *s + y;
    *c = (t - *s) - y;
    *s = t;
}

// out: the network outputs of this step, row p * live + (i - imin) (one per
// path and live rate), or, for the vector head (outputs > 0), row p column i - 1.
__global__ void __launch_bounds__(kT) euler_kernel(const PathArgs a, const float *Ctab, float y_scale, int k,
                                                    uint64_t chunk_first, int Pc, float *state,
                                                    const float *out, int outputs, int out_t, double *acc)
{
    __shared__ double red[kT / 32][64][2];
    const int n = a.n, s = a.s, ns = a.ns, imin = k / s + 1, live = n - imin + 1;
    const int p = blockIdx.x * kT + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool mat = (k + 1) % s == 0;
    const uint64_t lp = chunk_first + (uint64_t)p;
    const bool active = p < Pc && lp < a.paths;
    if (p < Pc) {
        uint64_t sidx = ~0ull;
        if (a.snap != nullptr && active && lp % a.snap_stride == 0 && lp / a.snap_stride < a.n_snap)
            sidx = lp / a.snap_stride;
        const float dH = draw_increment(a, a.first_path + lp, (uint32_t)k);
        const float h = a.h;
        // Rates in batches of 4: every load of a batch is issued before its
        // stores (the pointers do not alias), so the memory latencies overlap.
        const float *__restrict__ cr = Ctab + (size_t)k * n;
        const float4 *__restrict__ rr = a.row + (size_t)k * n;
        const float *__restrict__ op = out;
        float *__restrict__ sp = state;
        for (int i0 = n; i0 >= imin; i0 -= 4) {
            float o[4], zs[4], c[4], lam[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 - u;
                if (i < imin) break;
                const size_t oi = outputs > 0 ? (out_t ? (size_t)(i - 1) * Pc + p : (size_t)p * outputs + (i - 1))
                                              : (size_t)p * live + (i - imin);
                o[u] = op[oi];
                zs[u] = sp[(size_t)(i - 1) * Pc + p];
                c[u] = cr[i - 1];
                lam[u] = rr[i - 1].x;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 - u;
                if (i < imin) break;
                const float A = c[u] + y_scale * o[u];
                const float z = zs[u] + fmaf(lam[u], dH, -A * h);
                sp[(size_t)(i - 1) * Pc + p] = z;
                if (mat && sidx != ~0ull)
                    a.snap[((size_t)(imin - 1) * n + (i - 1)) * a.snap_pitch + sidx] = z + a.Z0[i - 1];
            }
        }
    }
    if (!mat) return;
    const int m = imin;
    double Pp = 1.0, Sp = 1.0;
    float Lm = 0.0f;
    if (p < Pc)
        maturity_products(a, m, [&](int i) { return state[(size_t)(i - 1) * Pc + p] + a.Z0[i - 1]; }, Pp, Sp, Lm);
    for (int q = 0; q < ns; ++q) {
        const float K = a.strikes[(size_t)(m - 1) * ns + q];
        const double pay = active ? payoff(a, Pp, Sp, Lm, K) : 0.0;
        const double s1 = warp_sum(pay), s2 = warp_sum(pay * pay);
        if (lane == 0) {
            red[warp][q][0] = s1;
            red[warp][q][1] = s2;
        }
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < kT / 32; ++w) {
            s1 += red[w][threadIdx.x][0];
            s2 += red[w][threadIdx.x][1];
        }
        double *c = acc + 4 * ((size_t)blockIdx.x * n * ns + (size_t)(m - 1) * ns + threadIdx.x);
        kahan_add(c + 0, c + 1, s1);
        kahan_add(c + 2, c + 3, s2);
    }
}

__global__ void acc_to_partials(const double *acc, size_t cells, double *partials)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cells) return;
    partials[2 * e + 0] = acc[4 * e + 0];
    partials[2 * e + 1] = acc[4 * e + 2];
}

}  // namespace

int mlp_layered_threads() { return kT; }

int launch_mlp_features(const PathArgs &a, const MlpScales &sc, int k, int Pc, const float *state, void *X,
                        int in_pad, int head, cudaStream_t st)
{
    if (head) {
        if (in_pad % 8) return (int)cudaErrorInvalidValue;
        const size_t smem = sizeof(float) * (size_t)a.n * (kFV + 1);
        feat_vec_kernel<<<(Pc + kFV - 1) / kFV, kT, smem, st>>>(a, sc, k, Pc, state,
                                                                 static_cast<__nv_bfloat16 *>(X), in_pad);
        return (int)cudaGetLastError();
    }
    const int live = a.n - (k / a.s + 1) + 1;
    const size_t rows = (size_t)Pc * live;
    feat_kernel<<<(unsigned)((rows + kT - 1) / kT), kT, 0, st>>>(a, sc, k, Pc, state,
                                                                  static_cast<__nv_bfloat16 *>(X), in_pad);
    return (int)cudaGetLastError();
}

int launch_mlp_euler(const PathArgs &a, const float *Ctab, float y_scale, int k, uint64_t chunk_first, int Pc,
                     float *state, const float *out, int outputs, int out_t, double *acc, cudaStream_t st)
{
    if (a.ns > 64) return (int)cudaErrorInvalidValue;
    euler_kernel<<<(Pc + kT - 1) / kT, kT, 0, st>>>(a, Ctab, y_scale, k, chunk_first, Pc, state, out, outputs,
                                                    out_t, acc);
    return (int)cudaGetLastError();
}

int launch_mlp_acc_to_partials(const double *acc, size_t cells, double *partials, cudaStream_t st)
{
    acc_to_partials<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(acc, cells, partials);
    return (int)cudaGetLastError();
}

}  // namespace lll
