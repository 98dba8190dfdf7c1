// lll_paths_tenor.cu -- tenor-parallel path kernels: G lanes share one path,
// each lane owning a contiguous block of its rates.
//
// Section 3.1-3.2 of the paper: the Picard iterate Z^(1) of Eq. (Picard-2)
// depends on the driving Levy path only, so the drift of Eq. (bdrift) lets
// every (path, tenor) evolve on its own.  Here lane g of a G-lane group owns
// the rates hi_g = n - g r down to lo_g = n - (g+1) r + 1 (r rates per lane,
// lane 0 the top block).  Per Euler step k every lane
//   1. takes the shared increment Delta H_k (lane k mod G of the group drew it),
//   2. forms the weights w_l = delta L_l / (1 + delta L_l) of its own rates:
//      PICARD from Z^(1)_l(t_k) = Z_l(0) + D0_l(t_k) + int_0^{t_k} lambda_l dH,
//      FULL from its own simulated Z_l(t_k) (left-point Euler: the drift of
//      every rate of step k reads the state at t_k),
//   3. multiplies the beta factors of its block, B_j = prod_{l in block}
//      (1 + w_l E_lj), for every quadrature node j,
//   4. takes the exclusive product of the blocks above it, Pre_j = prod_{g' < g}
//      B_j(g'), by a multiplicative scan over the group's lanes (shuffles), so
//      prod_{l > i} (1 + w_l E_lj) = Pre_j * prod_{l in block, l > i}(...) for
//      every rate i of the block,
//   5. sweeps its block from the top carrying P~_j = c_j Pre_j prod(...):
//      u = E_ij P~_j, A_i += u, P~_j += w_i u, so A_i = K_i + sum_j u (the
//      compensator of Eq. (LIBOR-drift-PT) with c_j = W_j / x_j^2), and
//      applies the Euler step of Eq. (log-LIB-SDE-2) to its own rates.
// No lane reads another lane's state: only the node products B_j cross lanes,
// and in the Picard scheme those are functions of the H path alone.
// At T_m the product prod_{l>m}(1 + delta L_l(T_m)) of the caplet numeraire of
// Eq. (caplet) is a product over the lanes (shuffles); the lane owning rate m
// forms the payoffs, reduced over the block into FP64 Kahan accumulators as
// in lll_paths.cu.
//
// Cost against the one-lane sweep (3 FP32 lane-ops per (node, live rate)):
// steps 3 and 5 take 2 + 3, and the scan adds (log2 G + 1) shuffles per node
// and lane and step.  The mapping gives G times as many threads per path, so
// it pays where paths are few (a single term structure of 2^12 paths fills a
// small fraction of the GPU with one thread per path).
//
// Layout: the live E rows of step k are staged into shared memory (cp.async,
// double-buffered across steps) with a row pitch of Q/4 + 1 float4 so that
// the G lanes of a group, each at its own rate, read different banks; per-path
// state (log-rate offsets, Picard's integrals, weights) stays in shared memory
// for the tile's lifetime.  Caplets only (swaptions need the one-lane kernel).
#include <cuda_runtime.h>

#include "lll_device.cuh"
#include "lll_internal.h"

namespace lll {
namespace {

constexpr int kTenorThreads = 128;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ float weight_of(float x)
{
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    return r;
}

__device__ __forceinline__ void kahan_add(double *s, double *c, double x)
{
    const double y = x - *c;
    const double t = *s + y;
    *c = (t - *s) - y;
    *s = t;
}

__host__ __device__ inline size_t a16(size_t v) { return (v + 15) & ~size_t(15); }

// Shared-memory plan (bytes); PB = paths per block, pitch PB + 1 floats.
struct TenorSmem {
    float4 *tab;  // [2][n][Q4 + 1]
    float4 *row;  // [2][n]: lambda, K, D0, b0 h
    float2 *cn;   // [QP / 2]
    float *c0;    // [n]
    float *sa;    // [n][PB + 1]: FULL z offset; PICARD int lambda dH
    float *sb;    // [n][PB + 1]: PICARD drift integral
    float *sw;    // [n][PB + 1]: weights of the step
    double *bsum; // [n * ns][4]
    double *red;  // [warps][ns] 16-byte slots (caplet_warp_sums)
};

__host__ __device__ inline size_t tenor_smem_bytes(int QP, int n, int ns, int T, int G)
{
    const int PB = T / G;
    size_t b = 0;
    b += a16(sizeof(float4) * 2 * (size_t)n * (QP / 4 + 1));
    b += a16(sizeof(float4) * 2 * (size_t)n);
    b += a16(sizeof(float) * (size_t)QP);
    b += a16(sizeof(float) * (size_t)n);
    b += 3 * a16(sizeof(float) * (size_t)n * (PB + 1));
    b += a16(sizeof(double) * 4 * (size_t)n * ns);
    b += a16(sizeof(double) * 2 * (size_t)(T / 32) * ns);
    return b;
}

__device__ inline TenorSmem tenor_carve(unsigned char *base, int QP, int n, int ns, int T, int G)
{
    const int PB = T / G;
    TenorSmem s;
    size_t o = 0;
    s.tab = reinterpret_cast<float4 *>(base + o);
    o += a16(sizeof(float4) * 2 * (size_t)n * (QP / 4 + 1));
    s.row = reinterpret_cast<float4 *>(base + o);
    o += a16(sizeof(float4) * 2 * (size_t)n);
    s.cn = reinterpret_cast<float2 *>(base + o);
    o += a16(sizeof(float) * (size_t)QP);
    s.c0 = reinterpret_cast<float *>(base + o);
    o += a16(sizeof(float) * (size_t)n);
    s.sa = reinterpret_cast<float *>(base + o);
    o += a16(sizeof(float) * (size_t)n * (PB + 1));
    s.sb = reinterpret_cast<float *>(base + o);
    o += a16(sizeof(float) * (size_t)n * (PB + 1));
    s.sw = reinterpret_cast<float *>(base + o);
    o += a16(sizeof(float) * (size_t)n * (PB + 1));
    s.bsum = reinterpret_cast<double *>(base + o);
    o += a16(sizeof(double) * 4 * (size_t)n * ns);
    s.red = reinterpret_cast<double *>(base + o);
    return s;
}

// Stage the live rows of step k (rates imin..n) into buffer b at row index
// rate - 1 (pitch Q4 + 1 float4).
template <int QP>
__device__ __forceinline__ void stage_step(const PathArgs &a, const TenorSmem &sm, int k, int b)
{
    constexpr int Q4 = QP / 4;
    const int n = a.n;
    const int imin = k / a.s + 1;
    const int cnt = n - imin + 1;
    const size_t r0 = (size_t)k * n + (imin - 1);
    const float4 *src = a.tab + r0 * Q4;
    float4 *dst = sm.tab + ((size_t)b * n + (imin - 1)) * (Q4 + 1);
    for (int e = threadIdx.x; e < cnt * Q4; e += blockDim.x) {
        const int rr = e / Q4, j4 = e - rr * Q4;
        cp_async16(dst + (size_t)rr * (Q4 + 1) + j4, src + e);
    }
    for (int e = threadIdx.x; e < cnt; e += blockDim.x)
        cp_async16(sm.row + (size_t)b * n + (imin - 1) + e, a.row + r0 + e);
}

template <int SCHEME, int QP, int G>
__global__ void __launch_bounds__(kTenorThreads) tenor_kernel(const PathArgs a, int r)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int Q2 = QP / 2, Q4 = QP / 4;
    constexpr unsigned FULLMASK = 0xffffffffu;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int PB = T / G, PP = PB + 1;
    const int p = tid / G, g = tid % G, gbase = lane & ~(G - 1);
    const int n = a.n, s = a.s, S = a.S, ns = a.ns;
    const float h = a.h;
    const TenorSmem sm = tenor_carve(smem_raw, QP, n, ns, T, G);
    for (int e = tid; e < n; e += T) sm.c0[e] = a.c0[e];
    for (int e = tid; e < QP; e += T) reinterpret_cast<float *>(sm.cn)[e] = a.cn[e];
    for (int e = tid; e < 4 * n * ns; e += T) sm.bsum[e] = 0.0;
    const int hi = n - g * r;                 // top rate of this lane's block (< 1: none)
    const int lo = max(1, n - (g + 1) * r + 1);
    const uint64_t ntiles = (a.paths + PB - 1) / PB;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t lp = tile * PB + p;
        const bool active = lp < a.paths;
        const uint64_t pid = a.first_path + lp;
        uint64_t sidx = ~0ull;
        if (a.snap != nullptr && active && lp % a.snap_stride == 0 && lp / a.snap_stride < a.n_snap)
            sidx = lp / a.snap_stride;
        for (int i = lo; i <= hi; ++i) {
            sm.sa[(i - 1) * PP + p] = 0.0f;
            sm.sb[(i - 1) * PP + p] = 0.0f;
        }
        __syncthreads(); // the previous tile's readers of both table buffers are done
        stage_step<QP>(a, sm, 0, 0);
        cp_commit();
        float dh_mine = 0.0f;

        for (int k = 0; k < S; ++k) {
            const int buf = k & 1;
            const int imin = k / s + 1;
            const bool mat = (k + 1) % s == 0;
            __syncthreads(); // buffer buf ^ 1 (read at step k - 1) is free
            if (k + 1 < S) stage_step<QP>(a, sm, k + 1, buf ^ 1);
            cp_commit();
            // increments: lane g draws step k + g once every G steps
            if (k % G == 0) {
                const int kk = k + g;
                dh_mine = (active && kk < S) ? draw_increment(a, pid, (uint32_t)kk) : 0.0f;
            }
            const float dH = __shfl_sync(FULLMASK, dh_mine, gbase + (k % G));
            cp_wait_1();
            __syncthreads();

            const float4 *tb = sm.tab + (size_t)buf * n * (Q4 + 1);
            const float4 *rb = sm.row + (size_t)buf * n;
            const int bot = max(lo, imin);
            // 2. weights of the own live rates
            for (int i = bot; i <= hi; ++i) {
                const float st = sm.sa[(i - 1) * PP + p];
                const float x = sm.c0[i - 1] + (SCHEME == PICARD ? rb[i - 1].z + st : st);
                sm.sw[(i - 1) * PP + p] = weight_of(x);
            }
            // 3. block products of the beta factors
            float2 B[Q2];
#pragma unroll
            for (int j = 0; j < Q2; ++j) B[j] = make_float2(1.0f, 1.0f);
            for (int i = bot; i <= hi; ++i) {
                const float w = sm.sw[(i - 1) * PP + p];
                const float2 w2 = make_float2(w, w), one = make_float2(1.0f, 1.0f);
                const float4 *tr = tb + (size_t)(i - 1) * (Q4 + 1);
#pragma unroll
                for (int j4 = 0; j4 < Q4; ++j4) {
                    const float4 v = tr[j4];
                    B[2 * j4] = __fmul2_rn(B[2 * j4], __ffma2_rn(w2, make_float2(v.x, v.y), one));
                    B[2 * j4 + 1] = __fmul2_rn(B[2 * j4 + 1], __ffma2_rn(w2, make_float2(v.z, v.w), one));
                }
            }
            // 4. exclusive product over the blocks above (lanes g' < g of the group)
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
#pragma unroll
                for (int j = 0; j < Q2; ++j) {
                    const float tx = __shfl_up_sync(FULLMASK, B[j].x, d, G);
                    const float ty = __shfl_up_sync(FULLMASK, B[j].y, d, G);
                    if (g >= d) B[j] = __fmul2_rn(B[j], make_float2(tx, ty));
                }
            }
#pragma unroll
            for (int j = 0; j < Q2; ++j) {
                const float tx = __shfl_up_sync(FULLMASK, B[j].x, 1, G);
                const float ty = __shfl_up_sync(FULLMASK, B[j].y, 1, G);
                const float2 pre = g ? make_float2(tx, ty) : make_float2(1.0f, 1.0f);
                B[j] = __fmul2_rn(sm.cn[j], pre); // P~_j = c_j Pre_j
            }
            // 5. sweep of the own block from the top, and the Euler step
            for (int i = hi; i >= bot; --i) {
                const float4 rc = rb[i - 1]; // lambda, K, D0, b0 h
                const float w = sm.sw[(i - 1) * PP + p];
                const float2 w2 = make_float2(w, w);
                const float4 *tr = tb + (size_t)(i - 1) * (Q4 + 1);
                float2 acc[4];
#pragma unroll
                for (int j4 = 0; j4 < Q4; ++j4) {
                    const float4 v = tr[j4];
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        const int j = 2 * j4 + hf;
                        const float2 e2 = hf ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
                        const float2 u = __fmul2_rn(e2, B[j]);
                        acc[j & 3] = (j < 4) ? u : __fadd2_rn(acc[j & 3], u);
                        B[j] = __ffma2_rn(w2, u, B[j]);
                    }
                }
                const float2 s2 = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
                const float bh = -(rc.y + (s2.x + s2.y)) * h;
                float *pa = sm.sa + (i - 1) * PP + p;
                if (SCHEME == PICARD) {
                    pa[0] = fmaf(rc.x, dH, pa[0]);           // int lambda dH
                    sm.sb[(i - 1) * PP + p] += bh;            // Picard drift integral
                } else {
                    pa[0] = pa[0] + fmaf(rc.x, dH, bh);
                }
            }

            if (mat) {
                const int m = imin;
                // log-rate offsets at T_m: z_l = sa (+ sb for Picard)
                auto zoff = [&](int i) {
                    float z = sm.sa[(i - 1) * PP + p];
                    if (SCHEME == PICARD) z += sm.sb[(i - 1) * PP + p];
                    return z;
                };
                float Pf = 1.0f;
                for (int i = hi; i >= max(lo, m + 1); --i) Pf *= fmaf(a.delta, expf(zoff(i) + a.Z0[i - 1]), 1.0f);
#pragma unroll
                for (int d = 1; d < G; d <<= 1) Pf *= __shfl_xor_sync(FULLMASK, Pf, d, G);
                const bool owner = m >= lo && m <= hi;
                const float Lm = owner ? expf(zoff(m) + a.Z0[m - 1]) : 0.0f;
                if (sidx != ~0ull)
                    for (int i = max(lo, m); i <= hi; ++i)
                        a.snap[((size_t)(m - 1) * n + (i - 1)) * a.snap_pitch + sidx] = zoff(i) + a.Z0[i - 1];
                for (int q = 0; q < ns; ++q) {
                    const float K = a.strikes[(size_t)(m - 1) * ns + q];
                    // the double-float sums inlined: as a call they raise this kernel's
                    // registers from 127 to 166
                    const float v = (owner && active) ? caplet_payoff(a, Pf, Lm, K) : 0.0f;
                    const float4 r = caplet_warp_sums_inline(DFloat{v, 0.0f}, df_square(v));
                    if (lane == 0) reinterpret_cast<float4 *>(sm.red)[(size_t)warp * ns + q] = r;
                }
                __syncthreads();
                if (tid < ns) {
                    double s1, s2;
                    block_payoff_sums(a, sm.red, T >> 5, ns, tid, s1, s2);
                    double *acc = sm.bsum + 4 * ((size_t)(m - 1) * ns + tid);
                    kahan_add(acc + 0, acc + 1, s1);
                    kahan_add(acc + 2, acc + 3, s2);
                }
            }
        }
        cp_wait_0();
    }
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += T) {
        out[2 * e + 0] = sm.bsum[4 * e + 0];
        out[2 * e + 1] = sm.bsum[4 * e + 2];
    }
}

typedef void (*TenorFn)(const PathArgs, int);

template <int SCHEME, int QP>
TenorFn pick_g(int G)
{
    switch (G) {
    case 4: return tenor_kernel<SCHEME, QP, 4>;
    case 8: return tenor_kernel<SCHEME, QP, 8>;
    case 16: return tenor_kernel<SCHEME, QP, 16>;
    case 32: return tenor_kernel<SCHEME, QP, 32>;
    default: return nullptr;
    }
}

template <int SCHEME>
TenorFn pick_qp(int QP, int G)
{
    switch (QP) {
    case 16: return pick_g<SCHEME, 16>(G);
    case 32: return pick_g<SCHEME, 32>(G);
    case 64: return pick_g<SCHEME, 64>(G);
    case 96: return pick_g<SCHEME, 96>(G);
    case 128: return pick_g<SCHEME, 128>(G);
    default: return nullptr;
    }
}

TenorFn pick_tenor(int scheme, int QP, int G)
{
    if (scheme == FULL) return pick_qp<FULL>(QP, G);
    if (scheme == PICARD) return pick_qp<PICARD>(QP, G);
    return nullptr;
}

}  // namespace

// Rates per lane: ceil(n / G), made odd so that the lanes of a group, each at
// its own rate, hit different shared-memory banks (row pitch Q/4 + 1 float4).
int tenor_rates_per_lane(int n, int G)
{
    int r = (n + G - 1) / G;
    if ((r & 1) == 0 && G > 1) ++r;
    return r;
}

bool tenor_kernel_supported(int scheme, int QP, int G) { return pick_tenor(scheme, QP, G) != nullptr; }

size_t tenor_kernel_smem(int QP, int n, int ns, int G) { return tenor_smem_bytes(QP, n, ns, kTenorThreads, G); }

int tenor_kernel_threads() { return kTenorThreads; }

int tenor_kernel_prepare(int scheme, int QP, int G, size_t smem, int *blocks_per_sm)
{
    TenorFn f = pick_tenor(scheme, QP, G);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kTenorThreads, smem);
}

int launch_tenor_kernel(int scheme, int QP, int G, int grid, size_t smem, cudaStream_t st, const PathArgs &a)
{
    TenorFn f = pick_tenor(scheme, QP, G);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, kTenorThreads, smem, st>>>(a, tenor_rates_per_lane(a.n, G));
    return (int)cudaGetLastError();
}

}  // namespace lll
