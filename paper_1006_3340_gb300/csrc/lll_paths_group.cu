// lll_paths_group.cu -- path kernels with G lanes per group of G paths (G = 2, 4).
//
// Same arithmetic as lll_paths.cu (the suffix sweep of the beta-factor
// products, Eq. (LIBOR-drift-PT) / (bdrift), the Euler step of
// Eq. (log-LIB-SDE-2) and the payoffs of Eq. (caplet)), mapped differently:
// lane t of a G-lane group owns path t of the group (its state, increment,
// weight w, Euler step and payoff) and sweeps the slice {t, t+G, t+2G,..} of
// the staged float4 table entries (four nodes each) for all G paths of the
// group, carrying the scaled products c_j P_j as the one-lane kernel does.  Each staged table
// value is therefore loaded once per lane and used for G paths, and the
// compensator A_i of each path is a sum over G lanes (a reduce-scatter by
// shuffles gives every lane the total of its own path).  The weights w of the
// G paths reach all lanes of the group by shuffles.
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

__host__ __device__ inline size_t a16(size_t v) { return (v + 15) & ~size_t(15); }

// The weights of the G paths of this lane's group, from each lane's own.
template <int G>
__device__ __forceinline__ void group_weights(float wown, int t, int gbase, float2 (&w2)[G])
{
    if constexpr (G == 2) {
        const float other = __shfl_xor_sync(0xffffffffu, wown, 1);
        const float w0 = t ? other : wown, w1 = t ? wown : other;
        w2[0] = make_float2(w0, w0);
        w2[1] = make_float2(w1, w1);
    } else {
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const float wq = __shfl_sync(0xffffffffu, wown, gbase + q);
            w2[q] = make_float2(wq, wq);
        }
    }
}

__host__ __device__ inline size_t group_smem_bytes(int QP, int n, int ns, int threads, int CH)
{
    size_t b = 0;
    b += a16(sizeof(float4) * 2 * (size_t)CH * (QP / 4));
    b += a16(sizeof(float4) * 2 * (size_t)CH);
    b += a16(sizeof(float) * (size_t)QP);
    b += a16(sizeof(float) * (size_t)n);
    b += a16(sizeof(double) * 4 * (size_t)n * ns);
    b += a16(sizeof(double) * 2 * (size_t)(threads / 32) * ns);
    return b;
}

template <int QP>
__device__ __forceinline__ void stage(const PathArgs &a, float4 *tab, float4 *row, int k, int c, int b)
{
    const int n = a.n, CH = a.chunk_rows;
    const int imin = k / a.s + 1;
    const int itop = n - c * CH;
    const int ibot = max(imin, itop - CH + 1);
    const int cnt = itop - ibot + 1;
    const size_t r0 = (size_t)k * n + (ibot - 1);
    constexpr int Q4 = QP / 4;
    const float4 *src = a.tab + r0 * Q4;
    float4 *dst = tab + (size_t)b * CH * Q4;
    for (int e = threadIdx.x; e < cnt * Q4; e += blockDim.x) cp_async16(dst + e, src + e);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) cp_async16(row + b * CH + e, a.row + r0 + e);
}

// SCHEME: FULL or PICARD; QP: padded node count (multiple of 16); G: lanes per
// group = paths per group (2 or 4).
template <int SCHEME, int QP, int G>
__global__ void __launch_bounds__(kMaxThreads, (QP <= 64 ? 2 : 1)) group_kernel(const PathArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int Q4 = QP / 4;     // float4 entries per table row (4 nodes each)
    constexpr int QL = Q4 / G;     // entries per lane
    constexpr int NST = (SCHEME == PICARD) ? 2 : 1;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = lane & (G - 1);               // lane within the group = owned path
    const int gbase = lane & ~(G - 1);          // first lane of the group
    const int n = a.n, s = a.s, S = a.S, ns = a.ns, CH = a.chunk_rows;
    float4 *stab, *srow;
    float *sc0, *scn;
    double *bsum, *red;
    {
        size_t o = 0;
        stab = reinterpret_cast<float4 *>(smem_raw + o); o += a16(sizeof(float4) * 2 * (size_t)CH * Q4);
        srow = reinterpret_cast<float4 *>(smem_raw + o); o += a16(sizeof(float4) * 2 * (size_t)CH);
        scn = reinterpret_cast<float *>(smem_raw + o); o += a16(sizeof(float) * (size_t)QP);
        sc0 = reinterpret_cast<float *>(smem_raw + o); o += a16(sizeof(float) * (size_t)n);
        bsum = reinterpret_cast<double *>(smem_raw + o); o += a16(sizeof(double) * 4 * (size_t)n * ns);
        red = reinterpret_cast<double *>(smem_raw + o);
    }
    for (int e = tid; e < n; e += T) sc0[e] = a.c0[e];
    for (int e = tid; e < QP; e += T) scn[e] = a.cn[e];
    for (int e = tid; e < 4 * n * ns; e += T) bsum[e] = 0.0;

    // Block slot [NST][n][T]: column = 4 * gidx + t = tid, i.e. this lane's path.
    float *st = a.state + (size_t)blockIdx.x * NST * n * T + tid;
    const uint64_t TP = (uint64_t)T;  // one path per lane
    const uint64_t ntiles = (a.paths + TP - 1) / TP;
    const float h = a.h;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t lp = tile * TP + tid;
        const bool active = lp < a.paths;
        const uint64_t p = a.first_path + lp;
        uint64_t sidx = ~0ull;
        if (a.snap != nullptr && active && lp % a.snap_stride == 0 && lp / a.snap_stride < a.n_snap)
            sidx = lp / a.snap_stride;
        for (int l = 0; l < NST * n; ++l) st[(size_t)l * T] = 0.0f;

        __syncthreads();
        stage<QP>(a, stab, srow, 0, 0, 0);
        cp_commit();
        int buf = 0;

        for (int k = 0; k < S; ++k) {
            const int imin = k / s + 1;
            const int nch = (n - imin + CH) / CH;
            const bool mat = (k + 1) % s == 0;
            const float dH = draw_increment(a, p, (uint32_t)k);
            // P[q][2j + hf]: scaled product c P of path q of the group, node
            // pair hf of table entry G j + t
            float2 P[G][2 * QL];
#pragma unroll
            for (int j = 0; j < QL; ++j) {
                const float4 cj = reinterpret_cast<const float4 *>(scn)[G * j + t];
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    P[q][2 * j] = make_float2(cj.x, cj.y);
                    P[q][2 * j + 1] = make_float2(cj.z, cj.w);
                }
            }

            for (int c = 0; c < nch; ++c) {
                int nk = k, nc = c + 1;
                if (nc == nch) { nk = k + 1; nc = 0; }
                if (nk < S) stage<QP>(a, stab, srow, nk, nc, buf ^ 1);
                cp_commit();
                cp_wait_1();
                __syncthreads();

                const int itop = n - c * CH;
                const int ibot = max(imin, itop - CH + 1);
                const float4 *tb = stab + (size_t)buf * CH * Q4;
                const float4 *rb = srow + buf * CH;
                // This lane's state and the group's weights for the first row;
                // every row then prepares the next row's, so MUFU and shuffle
                // latency overlap with the current node sweep.
                float v0n = st[(size_t)(itop - 1) * T];
                float v1n = (NST == 2) ? st[(size_t)(n + itop - 1) * T] : 0.0f;
                float2 wn2[G];
                group_weights<G>(weight_of(sc0[itop - 1] + (SCHEME == PICARD ? rb[itop - ibot].z : 0.0f) + v0n),
                                 t, gbase, wn2);
                for (int i = itop; i >= ibot; --i) {
                    const int r = i - ibot;
                    const float4 rc = rb[r]; // lambda, K, D0, b0*h
                    const float v0 = v0n, v1 = v1n;
                    float2 w2[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) w2[q] = wn2[q];
                    if (i > ibot) {
                        v0n = st[(size_t)(i - 2) * T];
                        if (NST == 2) v1n = st[(size_t)(n + i - 2) * T];
                        group_weights<G>(weight_of(sc0[i - 2] + (SCHEME == PICARD ? rb[r - 1].z : 0.0f) + v0n),
                                         t, gbase, wn2);
                    }
                    float2 acc[G][2];
                    const float4 *tr = tb + (size_t)r * Q4 + t;
#pragma unroll
                    for (int j = 0; j < QL; ++j) {
                        const float4 v = tr[G * j];
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            const float2 e2 = hf ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
#pragma unroll
                            for (int q = 0; q < G; ++q) {
                                const float2 u = __fmul2_rn(e2, P[q][2 * j + hf]);
                                acc[q][hf] = (j == 0) ? u : __fadd2_rn(acc[q][hf], u);
                                P[q][2 * j + hf] = __ffma2_rn(w2[q], u, P[q][2 * j + hf]);
                            }
                        }
                    }
                    float part[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) {
                        const float2 s2 = __fadd2_rn(acc[q][0], acc[q][1]);
                        part[q] = s2.x + s2.y;
                    }
                    // reduce-scatter over the G lanes: lane t ends with the total of path t
                    if constexpr (G == 2) {
                        const float keep = t ? part[1] : part[0], send = t ? part[0] : part[1];
                        part[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
                    } else {
                        const bool hi = (t & 2) != 0;
                        const float s0 = hi ? part[0] : part[2], s1 = hi ? part[1] : part[3];
                        const float r0 = __shfl_xor_sync(0xffffffffu, s0, 2);
                        const float r1 = __shfl_xor_sync(0xffffffffu, s1, 2);
                        float k0 = hi ? part[2] : part[0], k1 = hi ? part[3] : part[1];
                        k0 += r0;
                        k1 += r1;
                        const bool odd = (t & 1) != 0;
                        const float sx = odd ? k0 : k1;
                        const float rx = __shfl_xor_sync(0xffffffffu, sx, 1);
                        part[0] = (odd ? k1 : k0) + rx;
                    }
                    const float bh = -(rc.y + part[0]) * h;
                    float *sp = st + (size_t)(i - 1) * T;
                    float znew;
                    if (SCHEME == PICARD) {
                        const float y = fmaf(rc.x, dH, v0);
                        const float d = v1 + bh;
                        sp[0] = y;
                        sp[(size_t)n * T] = d;
                        znew = y + d;
                    } else {
                        const float z = v0 + fmaf(rc.x, dH, bh);
                        sp[0] = z;
                        znew = z;
                    }
                    if (mat && sidx != ~0ull)
                        a.snap[((size_t)(imin - 1) * n + (i - 1)) * a.snap_pitch + sidx] = znew + a.Z0[i - 1];
                }
                __syncthreads();
                buf ^= 1;
            }

            if (mat) {
                const int m = imin;
                double Pp, Sp;
                float Lm;
                maturity_products(a, m, [&](int i) {
                    float z = st[(size_t)(i - 1) * T];
                    if (NST == 2) z += st[(size_t)(n + i - 1) * T];
                    return z + a.Z0[i - 1];
                }, Pp, Sp, Lm);
                for (int q = 0; q < ns; ++q) {
                    const float K = a.strikes[(size_t)(m - 1) * ns + q];
                    const size_t slot = (size_t)warp * ns + q;
                    if (a.product == 0) {
                        const float v[1] = {active ? caplet_payoff(a, (float)Pp, Lm, K) : 0.0f};
                        const float4 r = caplet_warp_sums(v);
                        if (lane == 0) reinterpret_cast<float4 *>(red)[slot] = r;
                    } else {
                        const double pay = active ? payoff(a, Pp, Sp, Lm, K) : 0.0;
                        const double s1 = warp_sum(pay);
                        const double s2 = warp_sum(pay * pay);
                        if (lane == 0) {
                            red[2 * slot + 0] = s1;
                            red[2 * slot + 1] = s2;
                        }
                    }
                }
                __syncthreads();
                if (tid < ns) {
                    double s1, s2;
                    block_payoff_sums(a, red, T >> 5, ns, tid, s1, s2);
                    double *acc = bsum + 4 * ((size_t)(m - 1) * ns + tid);
                    kahan_add(acc + 0, acc + 1, s1);
                    kahan_add(acc + 2, acc + 3, s2);
                }
                __syncthreads();
            }
        }
        cp_wait_0();
    }
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += T) {
        out[2 * e + 0] = bsum[4 * e + 0];
        out[2 * e + 1] = bsum[4 * e + 2];
    }
}

typedef void (*GroupFn)(const PathArgs);

template <int SCHEME, int G>
GroupFn pick_g(int QP)
{
    switch (QP) {
    case 16: return group_kernel<SCHEME, 16, G>;
    case 32: return group_kernel<SCHEME, 32, G>;
    case 64: return group_kernel<SCHEME, 64, G>;
    case 96: return group_kernel<SCHEME, 96, G>;
    case 128: return group_kernel<SCHEME, 128, G>;
    default: return nullptr;
    }
}

GroupFn pick_group(int scheme, int QP, int G)
{
    if (G == 2) {
        if (scheme == FULL) return pick_g<FULL, 2>(QP);
        if (scheme == PICARD) return pick_g<PICARD, 2>(QP);
    } else if (G == 4) {
        if (scheme == FULL) return pick_g<FULL, 4>(QP);
        if (scheme == PICARD) return pick_g<PICARD, 4>(QP);
    }
    return nullptr;
}

}  // namespace

bool group_kernel_supported(int scheme, int QP, int G) { return pick_group(scheme, QP, G) != nullptr; }

size_t group_kernel_smem(int QP, int n, int ns, int threads, int chunk_rows)
{
    return group_smem_bytes(QP, n, ns, threads, chunk_rows);
}

int group_kernel_prepare(int scheme, int QP, int G, size_t smem, int threads, int *blocks_per_sm)
{
    GroupFn f = pick_group(scheme, QP, G);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

int launch_group_kernel(int scheme, int QP, int G, int grid, int threads, size_t smem, cudaStream_t st,
                        const PathArgs &a)
{
    GroupFn f = pick_group(scheme, QP, G);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, threads, smem, st>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace lll
