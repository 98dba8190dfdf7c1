// lll_expand.cu -- the full Euler scheme with the drift expansions of Section 3
// (Eq. (drifta): A', Eq. (drifta2): A'') in place of the jump compensator.
//
// Eq. (product) expands prod_{l>i} (1 + w_l (e^{lambda_l x} - 1)); truncated
// after the first or second order, every term of the compensator is a
// combination of the jump cumulant kappa, so the drift needs no nodes:
//   A'_i  = K1_i + sum_{l>i} w_l K2_il
//   A''_i = A'_i + sum_{i<k<l} w_k w_l K3_ikl
// with K1_i = kappa(lambda_i), K2_il = kappa(lambda_i+lambda_l) - kappa(lambda_i)
// - kappa(lambda_l) and K3_ikl the seven-term inclusion-exclusion of
// kappa(lambda_i+lambda_k+lambda_l) (first-order bracket with the signs the
// expansion gives).  The tables are built in FP64 on the host per step and
// staged into shared memory; w_l = delta L_l / (1 + delta L_l) comes from the
// simulated rates at t_k (full-scheme coupling).  One thread carries one path
// through all steps; payoffs of Eq. (caplet) are reduced like in the path
// kernels (warps, then a fixed-order FP64 Kahan sum per block).
#include <cuda_runtime.h>

#include "lll_device.cuh"
#include "lll_internal.h"

namespace lll {
namespace {

constexpr int kT = 128;

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

// Tables of step k: K1 [n], K2 [n][n], K3 [n][n][n] (order 2), zero outside
// i < l resp. i < k < l.
template <int ORDER>
__global__ void __launch_bounds__(kT) expand_kernel(const PathArgs a, const float *K1, const float *K2,
                                                    const float *K3)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, s = a.s, S = a.S, ns = a.ns, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t n2 = (size_t)n * n, n3 = n2 * n;
    float *k1 = reinterpret_cast<float *>(smem_raw);
    float *k2 = k1 + n;
    float *k3 = k2 + n2;
    float *ws = k3 + (ORDER == 2 ? n3 : 0);               // [n][kT] weights of this step
    size_t nf = (size_t)n + n2 + (ORDER == 2 ? n3 : 0) + (size_t)n * kT;
    nf += nf & 1;                                          // 8-byte alignment of the doubles
    double *bsum = reinterpret_cast<double *>(k1 + nf);   // [n][ns][4]
    double *red = bsum + 4 * (size_t)n * ns;               // [warps][ns][2]
    for (int e = tid; e < 4 * n * ns; e += kT) bsum[e] = 0.0;
    float *st = a.state + (size_t)blockIdx.x * n * kT + tid;
    const uint64_t ntiles = (a.paths + kT - 1) / kT;
    const float h = a.h;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t lp = tile * kT + tid;
        const bool active = lp < a.paths;
        const uint64_t p = a.first_path + lp;
        uint64_t sidx = ~0ull;
        if (a.snap != nullptr && active && lp % a.snap_stride == 0 && lp / a.snap_stride < a.n_snap)
            sidx = lp / a.snap_stride;
        for (int l = 0; l < n; ++l) st[(size_t)l * kT] = 0.0f;
        for (int k = 0; k < S; ++k) {
            const int imin = k / s + 1;
            const bool mat = (k + 1) % s == 0;
            __syncthreads(); // previous step's readers of the tables are done
            for (size_t e = tid; e < (size_t)n; e += kT) k1[e] = K1[(size_t)k * n + e];
            for (size_t e = tid; e < n2; e += kT) k2[e] = K2[(size_t)k * n2 + e];
            if (ORDER == 2)
                for (size_t e = tid; e < n3; e += kT) k3[e] = K3[(size_t)k * n3 + e];
            const float dH = draw_increment(a, p, (uint32_t)k);
            for (int l = imin; l <= n; ++l) {
                const float L = __expf(a.c0[l - 1] + st[(size_t)(l - 1) * kT]); // delta L_l
                ws[(size_t)(l - 1) * kT + tid] = L / (1.0f + L);
            }
            __syncthreads();
            for (int i = n; i >= imin; --i) {
                const float *r2 = k2 + (size_t)(i - 1) * n;
                float A = k1[i - 1];
                for (int l = i + 1; l <= n; ++l) A = fmaf(ws[(size_t)(l - 1) * kT + tid], r2[l - 1], A);
                if (ORDER == 2) {
                    const float *r3 = k3 + (size_t)(i - 1) * n2;
                    for (int kk = i + 1; kk < n; ++kk) {
                        float inner = 0.0f;
                        for (int l = kk + 1; l <= n; ++l)
                            inner = fmaf(ws[(size_t)(l - 1) * kT + tid], r3[(size_t)(kk - 1) * n + (l - 1)], inner);
                        A = fmaf(ws[(size_t)(kk - 1) * kT + tid], inner, A);
                    }
                }
                float *sp = st + (size_t)(i - 1) * kT;
                const float z = sp[0] + fmaf(a.row[(size_t)k * n + (i - 1)].x, dH, -A * h);
                sp[0] = z;
                if (mat && sidx != ~0ull)
                    a.snap[((size_t)(imin - 1) * n + (i - 1)) * a.snap_pitch + sidx] = z + a.Z0[i - 1];
            }
            if (mat) {
                const int m = imin;
                double Pp, Sp;
                float Lm;
                maturity_products(a, m, [&](int i) { return st[(size_t)(i - 1) * kT] + a.Z0[i - 1]; }, Pp, Sp, Lm);
                for (int q = 0; q < ns; ++q) {
                    const float K = a.strikes[(size_t)(m - 1) * ns + q];
                    const double pay = active ? payoff(a, Pp, Sp, Lm, K) : 0.0;
                    const double s1 = warp_sum(pay), s2 = warp_sum(pay * pay);
                    if (lane == 0) {
                        red[((size_t)warp * ns + q) * 2 + 0] = s1;
                        red[((size_t)warp * ns + q) * 2 + 1] = s2;
                    }
                }
                __syncthreads();
                if (tid < ns) {
                    double s1 = 0.0, s2 = 0.0;
                    for (int wv = 0; wv < kT / 32; ++wv) {
                        s1 += red[((size_t)wv * ns + tid) * 2 + 0];
                        s2 += red[((size_t)wv * ns + tid) * 2 + 1];
                    }
                    double *acc = bsum + 4 * ((size_t)(m - 1) * ns + tid);
                    kahan_add(acc + 0, acc + 1, s1);
                    kahan_add(acc + 2, acc + 3, s2);
                }
            }
        }
    }
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += kT) {
        out[2 * e + 0] = bsum[4 * e + 0];
        out[2 * e + 1] = bsum[4 * e + 2];
    }
}

}  // namespace

int expand_threads() { return kT; }

size_t expand_smem(int order, int n, int ns)
{
    const size_t n2 = (size_t)n * n, n3 = n2 * n;
    size_t f = (size_t)n + n2 + (order == 2 ? n3 : 0) + (size_t)n * kT;
    f += f & 1; // 8-byte alignment of the doubles
    return 4 * f + 8 * (4 * (size_t)n * ns + (kT / 32) * (size_t)ns * 2);
}

int expand_occupancy(int order, size_t smem, int *blocks_per_sm)
{
    void (*f)(const PathArgs, const float *, const float *, const float *) =
        order == 2 ? expand_kernel<2> : expand_kernel<1>;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kT, smem);
}

int launch_expand(int order, int grid, size_t smem, cudaStream_t st, const PathArgs &a, const float *K1,
                  const float *K2, const float *K3)
{
    if (order == 2) expand_kernel<2><<<grid, kT, smem, st>>>(a, K1, K2, K3);
    else expand_kernel<1><<<grid, kT, smem, st>>>(a, K1, K2, K3);
    return (int)cudaGetLastError();
}

}  // namespace lll
