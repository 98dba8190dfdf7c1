// lll_paths_step.cu -- the Picard scheme with its Euler steps evaluated in
// parallel (step-parallel mapping, lll_set_mapping(LLL_MAP_STEP)).
//
// Section 3.1-3.2 of the paper: under the Picard iterate of Eq. (Picard-2)
// the drift of Eq. (bdrift) at t_k reads
//     Z^(1)_l(t_k) = Z_l(0) + D0_l(t_k) + int_0^{t_k} lambda_l dH,
// a function of the driving path alone, and the log-rate is
//     Z_i(T_m) = Z_i(0) + sum_{k < m s} [ b_i(t_k; Z^(1)(t_k)) h + lambda_i(t_k) Delta H_k ].
// No step needs the simulated state of an earlier one, so the steps of a path
// are independent once the prefix sums of lambda_l Delta H are known.  (The
// full scheme's drift reads the simulated Z(t_k) and has no such form.)
// A launch is five kernels over a chunk of paths:
//   sp_draw     Delta H_k for every (step, path)                  [S][P]
//   sp_scan_y   Y_l(k) = sum_{m<k} lambda_l(m) Delta H_m          [S][n][P]
//   sp_sweep    one thread per (step, path): the suffix sweep of lll_paths.cu
//               at t_k with w_l from Z^(1)_l(t_k), giving b_i(t_k) h [S][n][P]
//   sp_scan_d   D_i(T_m) = sum_{k < m s} b_i h; log L_i(T_m)       [n][n][P]
//   sp_payoff   caplet payoffs of Eq. (caplet) at every T_m, reduced per block
// followed by the fixed-order block sum of lll_tables.cu.  Each unit does the
// arithmetic of the one-lane Picard kernel in the same order (the same weight,
// the same node sweep, the same running sums), so the two agree to rounding of
// the payoff reduction.  The intermediate arrays cost about 4 (S + 2 S n + n^2)
// bytes per path, so paths go through in chunks; the mapping pays where paths
// are few (a single term structure of 2^12 paths) and the autotuner chooses it.
#include <cuda_runtime.h>

#include <algorithm>

#include "lll_device.cuh"
#include "lll_internal.h"

namespace lll {
namespace {

constexpr int kSpT = 128; // threads per block of every kernel here

__device__ __forceinline__ float weight_of(float x)
{
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    return r;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kSpT) sp_draw(const PathArgs a, uint64_t chunk_first, int Pc, float *dH)
{
    const size_t e = (size_t)blockIdx.x * kSpT + threadIdx.x;
    if (e >= (size_t)a.S * Pc) return;
    const int k = (int)(e / Pc), lp = (int)(e % Pc);
    dH[e] = draw_increment(a, a.first_path + chunk_first + lp, (uint32_t)k);
}

// thread (l, path): Y[k][l][p] = sum_{m<k} lambda_l(m) dH_m for k < l s.
// The running sum is a dependent chain, so the loads of eight steps are issued
// ahead of their additions (same operations in the same order): one load
// latency per eight steps instead of one per step.
__global__ void __launch_bounds__(kSpT) sp_scan_y(const PathArgs a, int Pc, const float *__restrict__ dH,
                                                  float *__restrict__ Y)
{
    constexpr int U = 8;
    const size_t e = (size_t)blockIdx.x * kSpT + threadIdx.x;
    const int n = a.n;
    if (e >= (size_t)n * Pc) return;
    const int l = (int)(e / Pc) + 1, lp = (int)(e % Pc);
    const int K = l * a.s;
    const float *lam = reinterpret_cast<const float *>(a.row + (l - 1)); // .x of row (k, l): + 4 k n
    float y = 0.0f;
    int k = 0;
    for (; k + U <= K; k += U) {
        float lv[U], dv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            lv[u] = __ldg(lam + (size_t)4 * (k + u) * n);
            dv[u] = __ldg(dH + (size_t)(k + u) * Pc + lp);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Y[((size_t)(k + u) * n + (l - 1)) * Pc + lp] = y;
            y = fmaf(lv[u], dv[u], y);
        }
    }
    for (; k < K; ++k) {
        Y[((size_t)k * n + (l - 1)) * Pc + lp] = y;
        y = fmaf(__ldg(lam + (size_t)4 * k * n), __ldg(dH + (size_t)k * Pc + lp), y);
    }
}

// block (path block, step k): the live E rows of step k in shared memory, one
// thread per path sweeping the live rates n .. imin as the one-lane kernel does.
template <int QP>
__global__ void __launch_bounds__(kSpT) sp_sweep(const PathArgs a, int Pc, const float *Y, float *Bh)
{
    constexpr int Q2 = QP / 2, Q4 = QP / 4;
    extern __shared__ __align__(16) unsigned char smem_sp[];
    const int n = a.n, k = blockIdx.y, imin = k / a.s + 1, live = n - imin + 1;
    float4 *tab = reinterpret_cast<float4 *>(smem_sp);           // [live][Q4]
    float4 *row = tab + (size_t)live * Q4;                        // [live]
    float2 *cn = reinterpret_cast<float2 *>(row + live);          // [Q2]
    float *c0 = reinterpret_cast<float *>(cn + Q2);               // [live]
    const size_t r0 = (size_t)k * n + (imin - 1);
    for (int e = threadIdx.x; e < live * Q4; e += kSpT) tab[e] = a.tab[r0 * Q4 + e];
    for (int e = threadIdx.x; e < live; e += kSpT) {
        row[e] = a.row[r0 + e];
        c0[e] = a.c0[imin - 1 + e];
    }
    for (int e = threadIdx.x; e < QP; e += kSpT) reinterpret_cast<float *>(cn)[e] = a.cn[e];
    __syncthreads();
    const int lp = blockIdx.x * kSpT + threadIdx.x;
    if (lp >= Pc) return;
    const float h = a.h;
    float2 P[Q2];
#pragma unroll
    for (int j = 0; j < Q2; ++j) P[j] = cn[j];
    const float *Yk = Y + (size_t)k * n * Pc + lp;
    float yn = Yk[(size_t)(n - 1) * Pc];
    for (int i = n; i >= imin; --i) {
        const int r = i - imin;
        const float4 rc = row[r]; // lambda, K, D0, b0 h
        const float w = weight_of(c0[r] + rc.z + yn);
        if (i > imin) yn = Yk[(size_t)(i - 2) * Pc];
        const float2 w2 = make_float2(w, w);
        const float4 *tr = tab + (size_t)r * Q4;
        float2 acc[4];
#pragma unroll
        for (int j4 = 0; j4 < Q4; ++j4) {
            const float4 v = tr[j4];
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int j = 2 * j4 + hf;
                const float2 e2 = hf ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
                const float2 u = __fmul2_rn(e2, P[j]);
                acc[j & 3] = (j < 4) ? u : __fadd2_rn(acc[j & 3], u);
                P[j] = __ffma2_rn(w2, u, P[j]);
            }
        }
        const float2 s2 = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
        Bh[((size_t)k * n + (i - 1)) * Pc + lp] = -(rc.y + (s2.x + s2.y)) * h;
    }
}

// thread (i, path): running sums of the drift and of lambda dH; at every
// maturity T_m (m <= i) the log-rate log L_i(T_m) into Zm[m-1][i-1][p].  The
// drift terms of sixteen steps are loaded ahead of their additions (same
// operations in the same order), as in sp_scan_y.
__global__ void __launch_bounds__(kSpT) sp_scan_d(const PathArgs a, int Pc, uint64_t chunk_first,
                                                  const float *__restrict__ dH, const float *__restrict__ Y,
                                                  const float *__restrict__ Bh, float *__restrict__ Zm)
{
    constexpr int U = 16;
    const size_t e = (size_t)blockIdx.x * kSpT + threadIdx.x;
    const int n = a.n, s = a.s;
    if (e >= (size_t)n * Pc) return;
    const int i = (int)(e / Pc) + 1, lp = (int)(e % Pc);
    const uint64_t gp = chunk_first + lp; // path index within the simulation
    uint64_t sidx = ~0ull;
    if (a.snap != nullptr && gp % a.snap_stride == 0 && gp / a.snap_stride < a.n_snap) sidx = gp / a.snap_stride;
    const int K = i * s;
    float d = 0.0f;
    for (int k0 = 0; k0 < K; k0 += U) {
        float b[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            b[u] = k0 + u < K ? __ldg(Bh + ((size_t)(k0 + u) * n + (i - 1)) * Pc + lp) : 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u;
            if (k >= K) break;
            d = d + b[u];
            if ((k + 1) % s == 0) {
                const int m = (k + 1) / s;
                // int lambda_i dH up to T_m: the stored prefix at step m s, or for the
                // last step of rate i the same update as the one-lane kernel's
                const size_t ki = ((size_t)k * n + (i - 1)) * Pc + lp;
                const float y = m < i ? __ldg(Y + ((size_t)(k + 1) * n + (i - 1)) * Pc + lp)
                                      : fmaf(a.row[(size_t)k * n + (i - 1)].x, __ldg(dH + (size_t)k * Pc + lp),
                                             __ldg(Y + ki));
                const float z = y + d + a.Z0[i - 1];
                Zm[((size_t)(m - 1) * n + (i - 1)) * Pc + lp] = z;
                if (sidx != ~0ull) a.snap[((size_t)(m - 1) * n + (i - 1)) * a.snap_pitch + sidx] = z;
            }
        }
    }
}

// block (path block, maturity m): caplet payoffs of the block's paths at T_m,
// reduced in fixed order into partials[block][m-1][q][2].
__global__ void __launch_bounds__(kSpT) sp_payoff(const PathArgs a, int Pc, uint64_t chunk_first, const float *Zm,
                                                  int block0, double *partials)
{
    __shared__ __align__(16) double red[kSpT / 32 * 64 * 2]; // [warp][strike] 16-byte slots
    const int n = a.n, ns = a.ns, m = blockIdx.y + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lp = blockIdx.x * kSpT + threadIdx.x;
    const bool active = lp < Pc && chunk_first + lp < a.paths;
    double Pp = 1.0, Sp = 1.0;
    float Lm = 0.0f;
    if (lp < Pc)
        maturity_products(a, m, [&](int i) { return Zm[((size_t)(m - 1) * n + (i - 1)) * Pc + lp]; }, Pp, Sp, Lm);
    for (int q = 0; q < ns; ++q) {
        const float K = a.strikes[(size_t)(m - 1) * ns + q];
        const size_t slot = (size_t)warp * ns + q;
        if (a.product == 0) {
            const float v[1] = {active ? caplet_payoff(a, (float)Pp, Lm, K) : 0.0f};
            const float4 r = caplet_warp_sums(v);
            if (lane == 0) reinterpret_cast<float4 *>(red)[slot] = r;
        } else {
            const double v = active ? payoff(a, Pp, Sp, Lm, K) : 0.0;
            const double s1 = warp_sum(v), s2 = warp_sum(v * v);
            if (lane == 0) {
                red[2 * slot + 0] = s1;
                red[2 * slot + 1] = s2;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double s1, s2;
        block_payoff_sums(a, red, kSpT / 32, ns, threadIdx.x, s1, s2);
        double *out = partials + ((size_t)(block0 + blockIdx.x) * n + (m - 1)) * ns * 2 + 2 * threadIdx.x;
        out[0] = s1;
        out[1] = s2;
    }
}

typedef void (*SweepFn)(const PathArgs, int, const float *, float *);

SweepFn pick_sweep(int QP)
{
    switch (QP) {
    case 16: return sp_sweep<16>;
    case 32: return sp_sweep<32>;
    case 64: return sp_sweep<64>;
    case 96: return sp_sweep<96>;
    case 128: return sp_sweep<128>;
    default: return nullptr;
    }
}

unsigned blocks_of(size_t count) { return (unsigned)((count + kSpT - 1) / kSpT); }

}  // namespace

bool step_kernels_supported(int QP, int ns) { return pick_sweep(QP) != nullptr && ns <= 64; }

size_t step_bytes_per_path(int n, int S) { return 4 * ((size_t)S + 2 * (size_t)S * n + (size_t)n * n); }

int step_blocks_per_chunk(int Pc) { return (int)blocks_of((size_t)Pc); }

size_t step_sweep_smem(int QP, int n)
{
    return sizeof(float4) * (size_t)n * (QP / 4) + sizeof(float4) * (size_t)n + sizeof(float) * QP +
           sizeof(float) * (size_t)n;
}

// One chunk of Pc paths starting at chunk_first (relative to a.first_path).
// scratch: dH [S][Pc], Y and Bh [S][n][Pc], Zm [n][n][Pc] (floats).
// Payoff partials go to blocks block0 .. block0 + step_blocks_per_chunk(Pc) - 1.
int launch_step_chunk(int QP, const PathArgs &a, uint64_t chunk_first, int Pc, float *dH, float *Y, float *Bh,
                      float *Zm, int block0, double *partials, cudaStream_t st)
{
    SweepFn sw = pick_sweep(QP);
    if (!sw || a.ns > 64) return (int)cudaErrorInvalidValue;
    const int n = a.n, S = a.S;
    sp_draw<<<blocks_of((size_t)S * Pc), kSpT, 0, st>>>(a, chunk_first, Pc, dH);
    sp_scan_y<<<blocks_of((size_t)n * Pc), kSpT, 0, st>>>(a, Pc, dH, Y);
    const size_t smem = step_sweep_smem(QP, n);
    cudaError_t e = cudaFuncSetAttribute(sw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    sw<<<dim3(blocks_of((size_t)Pc), S), kSpT, smem, st>>>(a, Pc, Y, Bh);
    sp_scan_d<<<blocks_of((size_t)n * Pc), kSpT, 0, st>>>(a, Pc, chunk_first, dH, Y, Bh, Zm);
    sp_payoff<<<dim3(blocks_of((size_t)Pc), n), kSpT, 0, st>>>(a, Pc, chunk_first, Zm, block0, partials);
    return (int)cudaGetLastError();
}

}  // namespace lll
