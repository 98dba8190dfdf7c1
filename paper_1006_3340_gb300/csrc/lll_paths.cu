// lll_paths.cu -- the Monte Carlo path kernels (full Euler, Picard, frozen drift).
//
// One thread carries one path through all n*s Euler steps of Eq. (log-LIB-SDE-2)
// (Section 3).  Per step k it draws the shared increment Delta H_k and sweeps
// the live rates i = n .. i_min (rate i lives while k < i*s), carrying, for
// every quadrature node x_j, the running product
//     P_j = prod_{l > i} (1 + w_l (e^{lambda_l x_j} - 1))
// of the beta factors of Eq. (Levy-LIBOR-beta).  The jump part of the drift of
// Eq. (LIBOR-drift-PT) is then
//     A_i = int [(e^{lambda_i x}-1) prod_{l>i} beta_l - lambda_i x] F(dx)
//         = K_i + sum_j E_ij (c_j P_j),
// with E_ij = e^{lambda_i x_j} - 1, c_j = W_j / x_j^2 and
// K_i = C_i - sum_j c_j E_ij, C_i = sum_j c_j (E_ij - lambda_i x_j) (FP64
// tables).  The sweep carries the scaled products P~_j = c_j P_j (P~_j = c_j
// at the first rate of a step), so a table row holds E_ij alone, and costs 3
// FP32 operations per (node, live rate), packed as f32x2:
//     u = E_ij P~_j,   A_i += u,   P~_j += w_i u.
//
//  * FULL   (Eq. (LIBOR-drift-PT)): w_l from the simulated Z_l(t_k).
//  * PICARD (Eq. (bdrift)):         w_l from Z^(1)_l(t_k) = Z_l(0) + D0_l(t_k)
//                                   + int_0^{t_k} lambda_l dH (Eq. (Picard-2)),
//                                   which depends on the H path only.
//  * FROZEN:                        L^0 = exp(Z^(1)): the drift is b(t_k; Z(0)).
//  * Brownian driver (no quadrature): b_i = -lambda_i^2/2 - lambda_i sum_{l>i} w_l lambda_l.
//
// At T_m (end of step m*s-1) the caplet payoff of Eq. (caplet),
//     delta B(0,T_N) prod_{l>m} (1 + delta L_l(T_m)) (L_m(T_m) - K)^+,
// is reduced over the block (warp shuffles in double-float FP32 pairs, then
// warps in fixed order in FP64) into FP64 Kahan accumulators; per-block partials are summed in fixed order by a
// second kernel, so results are run-to-run deterministic.
//
// Layout: the per-step table rows (k, i) of the live rates are staged into
// shared memory in chunks of chunk_rows rows by cp.async, double-buffered so
// the next chunk loads while the current one is swept.  Every thread of a
// block is at the same (k, i), so table reads are shared-memory broadcasts.
// Path state (offsets of log L from log L(0)) lives in a per-block global
// scratch slot [nst][n][threads] that stays L1/L2 resident; the grid is
// persistent (one wave of resident blocks looping over path tiles).
#include <cuda_runtime.h>

#include "lll_device.cuh"
#include "lll_internal.h"

namespace lll {
namespace {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// delta L / (1 + delta L) for x = log(delta L) (approximate ex2 and rcp: w only
// scales the state-dependent part of the compensator).
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

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct Smem {
    float4 *tab;  // [2][CH * QP/4]
    float4 *row;  // [2][CH]
    float2 *cn;   // [QP/2] c_j = W_j / x_j^2
    float *c0;    // [n]
    double *bsum; // [n * ns][4]: sum, comp, sumsq, comp
    double *red;  // [warps][ns] 16-byte slots (block_payoff_sums)
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t smem_bytes(int QP, int n, int ns, int threads, int CH)
{
    size_t b = 0;
    b += align16(sizeof(float4) * 2 * (size_t)CH * (QP / 4));
    b += align16(sizeof(float4) * 2 * (size_t)CH);
    b += align16(sizeof(float) * (size_t)QP);
    b += align16(sizeof(float) * (size_t)n);
    b += align16(sizeof(double) * 4 * (size_t)n * ns);
    b += align16(sizeof(double) * 2 * (size_t)(threads / 32) * ns);
    return b;
}

__device__ inline Smem carve(unsigned char *base, int QP, int n, int ns, int threads, int CH)
{
    Smem s;
    size_t o = 0;
    s.tab = reinterpret_cast<float4 *>(base + o);
    o += align16(sizeof(float4) * 2 * (size_t)CH * (QP / 4));
    s.row = reinterpret_cast<float4 *>(base + o);
    o += align16(sizeof(float4) * 2 * (size_t)CH);
    s.cn = reinterpret_cast<float2 *>(base + o);
    o += align16(sizeof(float) * (size_t)QP);
    s.c0 = reinterpret_cast<float *>(base + o);
    o += align16(sizeof(float) * (size_t)n);
    s.bsum = reinterpret_cast<double *>(base + o);
    o += align16(sizeof(double) * 4 * (size_t)n * ns);
    s.red = reinterpret_cast<double *>(base + o);
    return s;
}

// Stage the table rows of chunk c of step k (rates i in [ibot, itop]) into buffer b.
template <int QP>
__device__ __forceinline__ void issue_chunk(const PathArgs &a, const Smem &sm, int k, int c, int b)
{
    const int n = a.n, CH = a.chunk_rows;
    const int imin = k / a.s + 1;
    const int itop = n - c * CH;
    const int ibot = max(imin, itop - CH + 1);
    const int cnt = itop - ibot + 1;
    const size_t r0 = (size_t)k * n + (ibot - 1);
    if (QP > 0) {
        constexpr int Q4 = QP / 4;
        const float4 *src = a.tab + r0 * Q4;
        float4 *dst = sm.tab + (size_t)b * CH * Q4;
        for (int e = threadIdx.x; e < cnt * Q4; e += blockDim.x) cp_async16(dst + e, src + e);
    }
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) cp_async16(sm.row + b * CH + e, a.row + r0 + e);
}

// One tile of T*R paths of the simulation `a`: all Euler steps, payoffs
// accumulated into sm.bsum.  st: this thread's column of the block's state slot.
template <int SCHEME, int QP, int R>
__device__ __forceinline__ void run_tile(const PathArgs &a, const Smem &sm, float *st, uint64_t tile)
{
    constexpr int Q2 = QP > 0 ? QP / 2 : 1; // node pairs
    constexpr int Q4 = QP > 0 ? QP / 4 : 1; // table float4 entries per row
    constexpr int NST = (SCHEME == PICARD) ? 2 : 1;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.n, s = a.s, S = a.S, ns = a.ns, CH = a.chunk_rows;
    const size_t rs = (size_t)NST * n * T; // stride between the R paths of a thread
    const uint64_t TP = (uint64_t)T * R;   // paths per tile
    const float h = a.h;
    {
        uint64_t lp[R], p[R], sidx[R];
        bool active[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            lp[q] = tile * TP + (uint64_t)q * T + tid; // path index within this simulation
            active[q] = lp[q] < a.paths;
            p[q] = a.first_path + lp[q];
            sidx[q] = ~0ull; // snapshot slot of this path, if it is recorded
            if (a.snap != nullptr && active[q] && lp[q] % a.snap_stride == 0 &&
                lp[q] / a.snap_stride < a.n_snap)
                sidx[q] = lp[q] / a.snap_stride;
        }
        for (int l = 0; l < R * NST * n; ++l) st[(size_t)l * T] = 0.0f;

        __syncthreads(); // previous tile's readers of both buffers are done
        issue_chunk<QP>(a, sm, 0, 0, 0);
        cp_commit();
        int buf = 0;

        for (int k = 0; k < S; ++k) {
            const int imin = k / s + 1;
            const int nch = (n - imin + CH) / CH; // ceil((n - imin + 1) / CH)
            const bool mat = (k + 1) % s == 0;     // rate imin fixes at t_{k+1} = T_imin
            float dH[R];
#pragma unroll
            for (int q = 0; q < R; ++q) dH[q] = draw_increment(a, p[q], (uint32_t)k);

            // scaled products P~_j = c_j P_j, P = 1 above the top rate
            float2 P[R][Q2];
            if (QP > 0) {
#pragma unroll
                for (int j = 0; j < Q2; ++j) {
                    const float2 cj = sm.cn[j];
#pragma unroll
                    for (int q = 0; q < R; ++q) P[q][j] = cj;
                }
            }
            float scont[R];
#pragma unroll
            for (int q = 0; q < R; ++q) scont[q] = 0.0f;

            for (int c = 0; c < nch; ++c) {
                int nk = k, nc = c + 1;
                if (nc == nch) { nk = k + 1; nc = 0; }
                if (nk < S) issue_chunk<QP>(a, sm, nk, nc, buf ^ 1);
                cp_commit();
                cp_wait_1();
                __syncthreads();

                const int itop = n - c * CH;
                const int ibot = max(imin, itop - CH + 1);
                const float4 *tb = sm.tab + (size_t)buf * CH * Q4;
                const float4 *rb = sm.row + buf * CH;
                // state of the first row; each row prefetches the next one's
                // State and weight of the first row; every row then loads the
                // next row's state and computes its weight, so that the MUFU
                // latency of w overlaps with the current row's node sweep.
                float c0v[R], c1v[R], wn[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    c0v[q] = st[q * rs + (size_t)(itop - 1) * T];
                    c1v[q] = (NST == 2) ? st[q * rs + (size_t)(n + itop - 1) * T] : 0.0f;
                    if (SCHEME != FROZEN)
                        wn[q] = weight_of(sm.c0[itop - 1] + (SCHEME == PICARD ? rb[itop - ibot].z : 0.0f) + c0v[q]);
                }
                for (int i = itop; i >= ibot; --i) {
                    const int r = i - ibot;
                    const float4 rc = rb[r]; // lambda, K, D0, b0*h
                    float v0[R], v1[R], w[R];
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        v0[q] = c0v[q];
                        v1[q] = c1v[q];
                        w[q] = wn[q];
                    }
                    if (i > ibot) {
                        const float cxn = sm.c0[i - 2] + (SCHEME == PICARD ? rb[r - 1].z : 0.0f);
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            c0v[q] = st[q * rs + (size_t)(i - 2) * T];
                            if (NST == 2) c1v[q] = st[q * rs + (size_t)(n + i - 2) * T];
                            if (SCHEME != FROZEN) wn[q] = weight_of(cxn + c0v[q]);
                        }
                    }
                    float bh[R];
                    if (SCHEME == FROZEN) {
#pragma unroll
                        for (int q = 0; q < R; ++q) bh[q] = rc.w;
                    } else if (QP > 0) {
                        const float4 *tr = tb + (size_t)r * Q4;
                        float2 acc[R][4];
                        float2 w2[R];
#pragma unroll
                        for (int q = 0; q < R; ++q) w2[q] = make_float2(w[q], w[q]);
#pragma unroll
                        for (int j4 = 0; j4 < Q4; ++j4) {
                            const float4 v = tr[j4];
#pragma unroll
                            for (int hf = 0; hf < 2; ++hf) {
                                const int j = 2 * j4 + hf;
                                const float2 e2 = hf ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
#pragma unroll
                                for (int q = 0; q < R; ++q) {
                                    const float2 u = __fmul2_rn(e2, P[q][j]);
                                    acc[q][j & 3] = (j < 4) ? u : __fadd2_rn(acc[q][j & 3], u);
                                    P[q][j] = __ffma2_rn(w2[q], u, P[q][j]);
                                }
                            }
                        }
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            const float2 s2 = __fadd2_rn(__fadd2_rn(acc[q][0], acc[q][1]), __fadd2_rn(acc[q][2], acc[q][3]));
                            bh[q] = -(rc.y + (s2.x + s2.y)) * h;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            bh[q] = (-0.5f * rc.x * rc.x - rc.x * scont[q]) * h;
                            scont[q] = fmaf(w[q], rc.x, scont[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        float *sp = st + q * rs + (size_t)(i - 1) * T;
                        float znew;
                        if (SCHEME == PICARD) {
                            const float y = fmaf(rc.x, dH[q], v0[q]); // int lambda dH
                            const float d = v1[q] + bh[q];            // Picard drift integral
                            sp[0] = y;
                            sp[(size_t)n * T] = d;
                            znew = y + d;
                        } else {
                            const float z = v0[q] + fmaf(rc.x, dH[q], bh[q]);
                            sp[0] = z;
                            znew = z;
                        }
                        if (mat && sidx[q] != ~0ull)
                            a.snap[((size_t)(imin - 1) * n + (i - 1)) * a.snap_pitch + sidx[q]] = znew + a.Z0[i - 1];
                    }
                }
                __syncthreads();
                buf ^= 1;
            }

            if (mat) {
                const int m = imin;
                // payoff quantities from the log-rates at T_m (state slot of this thread)
                double Pp[R], Sp[R];
                float Lm[R];
#pragma unroll
                for (int u = 0; u < R; ++u)
                    maturity_products(a, m, [&](int i) {
                        float z = st[u * rs + (size_t)(i - 1) * T];
                        if (NST == 2) z += st[u * rs + (size_t)(n + i - 1) * T];
                        return z + a.Z0[i - 1];
                    }, Pp[u], Sp[u], Lm[u]);
                for (int q = 0; q < ns; ++q) {
                    const float K = a.strikes[(size_t)(m - 1) * ns + q];
                    const size_t slot = (size_t)warp * ns + q;
                    if (a.product == 0) {
                        float v[R];
#pragma unroll
                        for (int u = 0; u < R; ++u) v[u] = active[u] ? caplet_payoff(a, (float)Pp[u], Lm[u], K) : 0.0f;
                        const float4 r = caplet_warp_sums(v);
                        if (lane == 0) reinterpret_cast<float4 *>(sm.red)[slot] = r;
                    } else {
                        double pay = 0.0, pay2 = 0.0;
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const double v = active[u] ? payoff(a, Pp[u], Sp[u], Lm[u], K) : 0.0;
                            pay += v;
                            pay2 += v * v;
                        }
                        const double s1 = warp_sum(pay);
                        const double s2 = warp_sum(pay2);
                        if (lane == 0) {
                            sm.red[2 * slot + 0] = s1;
                            sm.red[2 * slot + 1] = s2;
                        }
                    }
                }
                __syncthreads();
                if (tid < ns) {
                    double s1, s2;
                    block_payoff_sums(a, sm.red, T >> 5, ns, tid, s1, s2);
                    double *acc = sm.bsum + 4 * ((size_t)(m - 1) * ns + tid);
                    kahan_add(acc + 0, acc + 1, s1);
                    kahan_add(acc + 2, acc + 3, s2);
                }
                __syncthreads();
            }
        }
        cp_wait_0();
    }
}

// Register budget classes (resident warps hide shared-memory latency):
//   LB 0: up to 255 registers (node tables of 96 or 128 nodes),
//   LB 1: 128 registers, two 256-thread or four 128-thread blocks per SM,
//   LB 2: 102 registers, five blocks of at most 128 threads per SM.
template <int LB>
struct Bounds {
    static constexpr int threads = LB == 2 ? 128 : kMaxThreads;
    static constexpr int blocks = LB == 0 ? 1 : (LB == 1 ? 2 : 5);
};

template <int SCHEME, int QP, int R, int LB>
__global__ void __launch_bounds__(Bounds<LB>::threads, Bounds<LB>::blocks) path_kernel(const PathArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NST = (SCHEME == PICARD) ? 2 : 1;
    const int T = blockDim.x, tid = threadIdx.x;
    const int n = a.n, ns = a.ns;
    const Smem sm = carve(smem_raw, QP, n, ns, T, a.chunk_rows);
    for (int e = tid; e < n; e += T) sm.c0[e] = a.c0[e];
    for (int e = tid; e < QP; e += T) reinterpret_cast<float *>(sm.cn)[e] = a.cn[e];
    for (int e = tid; e < 4 * n * ns; e += T) sm.bsum[e] = 0.0;
    // This block's state slot: [R][NST][n][T]; thread tid owns column tid.
    float *st = a.state + (size_t)blockIdx.x * R * NST * n * T + tid;
    const uint64_t ntiles = (a.paths + (uint64_t)T * R - 1) / ((uint64_t)T * R);
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) run_tile<SCHEME, QP, R>(a, sm, st, tile);
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += T) {
        out[2 * e + 0] = sm.bsum[4 * e + 0];
        out[2 * e + 1] = sm.bsum[4 * e + 2];
    }
}

// Many independent term structures in one persistent launch.  The work is a
// list of items -- a range of consecutive tiles of one instance -- sorted by
// decreasing cost; every block claims the next item from a counter until the
// list is exhausted, so the longest items start first and the short ones fill
// the end (longest-processing-time-first list scheduling, Graham 1969).  Each
// item writes its payoff sums to its own segment, and a second kernel adds the
// segments of each instance in tile order, so the results do not depend on
// which block ran which item.  R paths per thread, as in path_kernel (a tile
// is T R paths).
template <int SCHEME, int QP, int R>
__global__ void __launch_bounds__(kMaxThreads) batch_kernel(const BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NST = (SCHEME == PICARD) ? 2 : 1;
    const int T = blockDim.x, tid = threadIdx.x;
    const Smem sm = carve(smem_raw, QP, b.n_max, b.ns_max, T, b.chunk_rows);
    float *st = b.state + (size_t)blockIdx.x * R * NST * b.n_max * T + tid;
    int cur = -1;
    __shared__ PathArgs sa; // the current instance's arguments
    __shared__ int claimed;
    const PathArgs *a = &sa;
    for (;;) {
        __syncthreads(); // the previous item's outputs are written, `claimed` read
        if (tid == 0) claimed = atomicAdd(b.next, 1);
        __syncthreads();
        const int it = claimed;
        if (it >= b.n_items) break;
        const int q = b.item_inst[it];
        if (q != cur) {
            cur = q;
            if (tid == 0) sa = b.desc[q];
            __syncthreads();
            for (int e = tid; e < a->n; e += T) sm.c0[e] = a->c0[e];
            for (int e = tid; e < QP; e += T) reinterpret_cast<float *>(sm.cn)[e] = a->cn[e];
        }
        for (int e = tid; e < 4 * a->n * a->ns; e += T) sm.bsum[e] = 0.0;
        const uint2 tr = b.item_tiles[it];
        for (uint32_t t = tr.x; t < tr.y; ++t) run_tile<SCHEME, QP, R>(*a, sm, st, t);
        __syncthreads();
        double *out = b.partials + b.seg_off[it];
        for (int e = tid; e < a->n * a->ns; e += T) {
            out[2 * e + 0] = sm.bsum[4 * e + 0];
            out[2 * e + 1] = sm.bsum[4 * e + 2];
        }
    }
}

typedef void (*KernelFn)(const PathArgs);

// Paths per thread: 2 shares every staged table load between two paths
// (halving shared-memory traffic per unit); compiled where the registers of
// two node arrays fit (padded Q <= 64).
// Budget by node count: <= 32 nodes and <= 128 threads: LB 2; <= 96 nodes:
// LB 1; more: LB 0.  Two paths per thread keep the full budget.
template <int SCHEME, int QP>
KernelFn pick_r(int R, int T)
{
    if (R == 1) {
        if constexpr (QP <= 32) {
            if (T <= 128) return path_kernel<SCHEME, QP, 1, 2>;
        }
        if constexpr (QP <= 96) return path_kernel<SCHEME, QP, 1, 1>;
        else return path_kernel<SCHEME, QP, 1, 0>;
    }
    if constexpr (QP <= 64) {
        if (R == 2) return path_kernel<SCHEME, QP, 2, 0>;
    }
    return nullptr;
}

template <int SCHEME>
KernelFn pick_qp(int QP, int R, int T)
{
    switch (QP) {
    case 0: return pick_r<SCHEME, 0>(R, T);
    case 16: return pick_r<SCHEME, 16>(R, T);
    case 32: return pick_r<SCHEME, 32>(R, T);
    case 64: return pick_r<SCHEME, 64>(R, T);
    case 96: return pick_r<SCHEME, 96>(R, T);
    case 128: return pick_r<SCHEME, 128>(R, T);
    default: return nullptr;
    }
}

KernelFn pick(int scheme, int QP, int R, int T)
{
    switch (scheme) {
    case FULL: return pick_qp<FULL>(QP, R, T);
    case PICARD: return pick_qp<PICARD>(QP, R, T);
    case FROZEN: return pick_r<FROZEN, 0>(R, T);
    default: return nullptr;
    }
}

typedef void (*BatchFn)(const BatchArgs);

template <int SCHEME>
BatchFn pick_batch_s(int QP, int R)
{
    if (R == 2) { // two paths per thread: compiled where the registers of two node arrays fit
        switch (QP) {
        case 16: return batch_kernel<SCHEME, 16, 2>;
        case 32: return batch_kernel<SCHEME, 32, 2>;
        case 64: return batch_kernel<SCHEME, 64, 2>;
        default: return nullptr;
        }
    }
    if (R != 1) return nullptr;
    switch (QP) {
    case 16: return batch_kernel<SCHEME, 16, 1>;
    case 32: return batch_kernel<SCHEME, 32, 1>;
    case 64: return batch_kernel<SCHEME, 64, 1>;
    case 96: return batch_kernel<SCHEME, 96, 1>;
    case 128: return batch_kernel<SCHEME, 128, 1>;
    default: return nullptr;
    }
}

BatchFn pick_batch(int scheme, int QP, int R)
{
    if (scheme == PICARD) return pick_batch_s<PICARD>(QP, R);
    if (scheme == FULL) return pick_batch_s<FULL>(QP, R);
    return nullptr;
}

}  // namespace

bool batch_kernel_supported(int scheme, int QP, int R) { return pick_batch(scheme, QP, R) != nullptr; }

int batch_kernel_prepare(int scheme, int QP, int R, size_t smem, int threads, int *blocks_per_sm)
{
    BatchFn f = pick_batch(scheme, QP, R);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

int launch_batch_kernel(int scheme, int QP, int R, int grid, int threads, size_t smem, cudaStream_t st,
                        const BatchArgs &b)
{
    BatchFn f = pick_batch(scheme, QP, R);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, threads, smem, st>>>(b);
    return (int)cudaGetLastError();
}

bool path_kernel_supported(int scheme, int QP, int R) { return pick(scheme, QP, R, kMaxThreads) != nullptr; }

size_t path_kernel_smem(int QP, int n, int ns, int threads, int chunk_rows)
{
    return smem_bytes(QP, n, ns, threads, chunk_rows);
}

int path_kernel_prepare(int scheme, int QP, int R, int threads, size_t smem)
{
    KernelFn f = pick(scheme, QP, R, threads);
    if (!f) return (int)cudaErrorInvalidValue;
    return (int)cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int path_kernel_occupancy(int scheme, int QP, int R, int threads, size_t smem, int *blocks_per_sm)
{
    KernelFn f = pick(scheme, QP, R, threads);
    if (!f) return (int)cudaErrorInvalidValue;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

int launch_path_kernel(int scheme, int QP, int R, int grid, int threads, size_t smem, cudaStream_t st,
                       const PathArgs &a)
{
    KernelFn f = pick(scheme, QP, R, threads);
    if (!f) return (int)cudaErrorInvalidValue;
    // The frozen kernel stages no node table; its QP argument is ignored.
    f<<<grid, threads, smem, st>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace lll
