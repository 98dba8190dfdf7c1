// lll_mlp_data.cu -- training data for the learned compensator.
//
// datagen_kernel: the full scheme (Eq. (LIBOR-drift-PT) with the quadrature
// compensator, same tables as the path kernels) simulated on its own paths,
// one thread per path.  At a few Euler steps per path, chosen by Philox, it
// records the log-rate offsets log L_m(t_k) - log L_m(0) of all rates and,
// for every live rate i, the target A_i - C_i = sum_j E_ij c_j (P_j - 1): the
// part of the compensator that depends on the later rates.  M_j = c_j (P_j - 1)
// is carried directly, M' = M + w E (c_j + M), so the small target keeps its
// relative accuracy in FP32.
// gather_kernel: a training batch of feature rows and scaled targets, drawn
// uniformly over records and, within a record, over its live rates.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lll_device.cuh"
#include "lll_internal.h"
#include "lll_mlp.h"

namespace lll {
namespace {

template <int QP>
__global__ void datagen_kernel(const PathArgs a, const float *Ctab, int R, uint32_t rec_key,
                               float *state, float *rec_u, float *rec_y, int *rec_k)
{
    constexpr int Q4 = QP / 4;
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.paths) return;
    const int n = a.n, s = a.s, S = a.S, N = n + 1;
    const float h = a.h;
    float *st = state + p; // [n][paths]
    const size_t pitch = a.paths;
    for (int l = 0; l < n; ++l) st[(size_t)l * pitch] = 0.0f;
    int ks[8];
    for (int r = 0; r < R; ++r) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)r, 0x9D3Au, (uint32_t)p, (uint32_t)(p >> 32)),
                                      rec_key, a.key1);
        ks[r] = (int)(w.x % (uint32_t)S);
    }
    for (int k = 0; k < S; ++k) {
        const int imin = k / s + 1;
        const float dH = draw_increment(a, a.first_path + p, (uint32_t)k);
        int slot[8], nrec = 0;
        for (int r = 0; r < R; ++r)
            if (ks[r] == k) slot[nrec++] = (int)(p * R + r);
        for (int q = 0; q < nrec; ++q) {
            float *u = rec_u + (size_t)slot[q] * N;
            u[0] = 0.0f;
            for (int m = 1; m <= n; ++m) u[m] = st[(size_t)(m - 1) * pitch];
            float *y = rec_y + (size_t)slot[q] * n;
            for (int m = 1; m < imin; ++m) y[m - 1] = 0.0f;
            rec_k[slot[q]] = k;
        }
        float4 M[Q4];
#pragma unroll
        for (int j = 0; j < Q4; ++j) M[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int i = n; i >= imin; --i) {
            const size_t row = (size_t)k * n + (i - 1);
            const float4 rc = __ldg(&a.row[row]);
            const float zoff = st[(size_t)(i - 1) * pitch];
            const float w = 1.0f / (1.0f + expf(-(a.c0[i - 1] + zoff)));
            float dep = 0.0f;
            const float4 *tr = a.tab + row * Q4;
            const float4 *cq = reinterpret_cast<const float4 *>(a.cn);
#pragma unroll
            for (int j = 0; j < Q4; ++j) {
                const float4 v = __ldg(&tr[j]), c = __ldg(&cq[j]);
                dep = fmaf(v.x, M[j].x, dep);
                dep = fmaf(v.y, M[j].y, dep);
                dep = fmaf(v.z, M[j].z, dep);
                dep = fmaf(v.w, M[j].w, dep);
                M[j].x = fmaf(w * v.x, c.x + M[j].x, M[j].x);
                M[j].y = fmaf(w * v.y, c.y + M[j].y, M[j].y);
                M[j].z = fmaf(w * v.z, c.z + M[j].z, M[j].z);
                M[j].w = fmaf(w * v.w, c.w + M[j].w, M[j].w);
            }
            for (int q = 0; q < nrec; ++q) rec_y[(size_t)slot[q] * n + (i - 1)] = dep;
            const float A = Ctab[row] + dep;
            st[(size_t)(i - 1) * pitch] = zoff + fmaf(rc.x, dH, -A * h);
        }
    }
}

// One training row per thread: features (t/T_N, i/n, lambda/lambda_ref, u_0..u_{N-1})
// padded with zeros to in_pad, and y = (A_i - C_i) / y_scale.
__global__ void gather_kernel(const float *rec_u, const float *rec_y, const int *rec_k, uint64_t nrec,
                              const double *lam, int n, int s, double delta, MlpScales sc, int in_pad,
                              int rows, uint32_t key0, uint32_t key1, uint32_t step,
                              __nv_bfloat16 *X, float *Y)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= rows) return;
    const int N = n + 1;
    const uint4 w = philox4x32_10(make_uint4(step, (uint32_t)b, 0x6A7Eu, 0u), key0, key1);
    const uint64_t slot = ((uint64_t)w.x << 32 | w.y) % nrec;
    const int k = rec_k[slot];
    const int imin = k / s + 1;
    const int i = imin + (int)(w.z % (uint32_t)(n - imin + 1));
    __nv_bfloat16 *xr = X + (size_t)b * in_pad;
    const double h = delta / s;
    xr[0] = __float2bfloat16((float)(k * h) * sc.t_scale);
    xr[1] = __float2bfloat16((float)i * sc.i_scale);
    xr[2] = __float2bfloat16((float)lam[(size_t)k * n + (i - 1)] * sc.lam_scale);
    for (int m = 0; m < N; ++m) xr[3 + m] = __float2bfloat16(rec_u[slot * N + m] * sc.u_scale);
    for (int c = 3 + N; c < in_pad; ++c) xr[c] = __float2bfloat16(0.0f);
    Y[b] = rec_y[slot * n + (i - 1)] / sc.y_scale;
}

// Vector head: one training row per recorded (path, step), drawn uniformly:
// features (t/T_N, u_0 .. u_{N-1}) padded to in_pad, targets y_i / y_scale for
// every rate (columns i - 1 < O; rates already fixed are masked by the loss
// through the row's step kr).
__global__ void gather_vec_kernel(const float *rec_u, const float *rec_y, const int *rec_k, uint64_t nrec, int n,
                                  int s, double delta, MlpScales sc, int in_pad, int O, int rows, uint32_t key0,
                                  uint32_t key1, uint32_t step, __nv_bfloat16 *X, float *Y, int *kr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= rows) return;
    const int N = n + 1;
    const uint4 w = philox4x32_10(make_uint4(step, (uint32_t)b, 0x7EC7u, 0u), key0, key1);
    const uint64_t slot = ((uint64_t)w.x << 32 | w.y) % nrec;
    const int k = rec_k[slot];
    __nv_bfloat16 *xr = X + (size_t)b * in_pad;
    const double h = delta / s;
    xr[0] = __float2bfloat16((float)(k * h) * sc.t_scale);
    for (int m = 0; m < N; ++m) xr[1 + m] = __float2bfloat16(rec_u[slot * N + m] * sc.u_scale);
    for (int c = 1 + N; c < in_pad; ++c) xr[c] = __float2bfloat16(0.0f);
    for (int o = 0; o < O; ++o) Y[(size_t)b * O + o] = o < n ? rec_y[slot * n + o] / sc.y_scale : 0.0f;
    kr[b] = k;
}

// Sum of squares and count of the recorded targets of live rates (per block).
__global__ void target_moments(const float *rec_y, const int *rec_k, uint64_t nrec, int n, int s,
                               double *part)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrec * n;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t slot = e / n;
        const int i = (int)(e % n) + 1;
        if (i >= rec_k[slot] / s + 1) acc += (double)rec_y[e] * rec_y[e];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace

int mlp_datagen(int QP, const PathArgs &a, const float *Ctab, int R, uint32_t rec_key, float *state,
                float *rec_u, float *rec_y, int *rec_k, cudaStream_t st)
{
    if (R < 1 || R > 8) return (int)cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((a.paths + 127) / 128);
    switch (QP) {
    case 16: datagen_kernel<16><<<grid, 128, 0, st>>>(a, Ctab, R, rec_key, state, rec_u, rec_y, rec_k); break;
    case 32: datagen_kernel<32><<<grid, 128, 0, st>>>(a, Ctab, R, rec_key, state, rec_u, rec_y, rec_k); break;
    case 64: datagen_kernel<64><<<grid, 128, 0, st>>>(a, Ctab, R, rec_key, state, rec_u, rec_y, rec_k); break;
    case 96: datagen_kernel<96><<<grid, 128, 0, st>>>(a, Ctab, R, rec_key, state, rec_u, rec_y, rec_k); break;
    case 128: datagen_kernel<128><<<grid, 128, 0, st>>>(a, Ctab, R, rec_key, state, rec_u, rec_y, rec_k); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int mlp_gather(const float *rec_u, const float *rec_y, const int *rec_k, uint64_t nrec, const double *lam,
               int n, int s, double delta, const MlpScales &sc, int in_pad, int rows, uint32_t key0,
               uint32_t key1, uint32_t step, void *X, float *Y, cudaStream_t st)
{
    gather_kernel<<<(rows + 127) / 128, 128, 0, st>>>(rec_u, rec_y, rec_k, nrec, lam, n, s, delta, sc,
                                                      in_pad, rows, key0, key1, step,
                                                      static_cast<__nv_bfloat16 *>(X), Y);
    return (int)cudaGetLastError();
}

int mlp_gather_vec(const float *rec_u, const float *rec_y, const int *rec_k, uint64_t nrec, int n, int s,
                   double delta, const MlpScales &sc, int in_pad, int O, int rows, uint32_t key0, uint32_t key1,
                   uint32_t step, void *X, float *Y, int *kr, cudaStream_t st)
{
    gather_vec_kernel<<<(rows + 127) / 128, 128, 0, st>>>(rec_u, rec_y, rec_k, nrec, n, s, delta, sc, in_pad, O,
                                                          rows, key0, key1, step,
                                                          static_cast<__nv_bfloat16 *>(X), Y, kr);
    return (int)cudaGetLastError();
}

int mlp_target_moments(const float *rec_y, const int *rec_k, uint64_t nrec, int n, int s, double *part,
                       int blocks, cudaStream_t st)
{
    target_moments<<<blocks, 256, 0, st>>>(rec_y, rec_k, nrec, n, s, part);
    return (int)cudaGetLastError();
}

}  // namespace lll
