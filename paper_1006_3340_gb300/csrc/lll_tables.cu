// lll_tables.cu -- FP64 precomputation on the GPU and the final reduction.
//
// tables_kernel: for every step k and rate l, the node table of the jump
//   compensator of Eq. (LIBOR-drift-PT): E_lj = e^{lambda_l(t_k) x_j} - 1
//   (rounded to FP32), the per-node factors c_j = W_j / x_j^2 (FP32), and the
//   constant K_l = C_l - sum_j fl32(E_lj c_j) with
//   C_l = sum_j W_j (E_lj - lambda_l x_j) / x_j^2, so that
//   A_l = K_l + sum_j E_lj (c_j P_j) reproduces C_l when P = 1 up to the FP32
//   sum.  C_l itself (the compensator with all later weights zero) is kept too.
// frozen_drift_kernel: the drift b(t_k, T_l; Z(0)) of Eq. (Picard-2), i.e.
//   Eq. (LIBOR-drift-PT) with L frozen at L(0), one block per step and one
//   thread per node, a fixed-order block sum per rate.
// prefix_kernel: D0_l(t_k) = sum_{m<k} b0_l(t_m) h, the deterministic drift
//   integral of Z^(1).
// finalize_kernel: sum of the per-block payoff partials in block order.
#include <cuda_runtime.h>

#include "lll_internal.h"

namespace lll {
namespace {

__global__ void tables_kernel(const double *lam, const double *x, const double *W, int n, int S,
                              int Q, int QP, float4 *tab, float *cn, float4 *row, float *Ctab)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    for (int j = idx; j < QP; j += gridDim.x * blockDim.x)
        cn[j] = (j < Q) ? (float)(W[j] / (x[j] * x[j])) : 0.0f;
    if (idx >= S * n) return;
    const double li = lam[idx];
    double C = 0.0, sa = 0.0;
    float *out = reinterpret_cast<float *>(tab + (size_t)idx * (QP / 4));
    for (int j = 0; j < QP; ++j) {
        float e = 0.0f;
        if (j < Q) {
            const double xj = x[j];
            const double ed = expm1(li * xj);
            const double inv = W[j] / (xj * xj);
            C += inv * (ed - li * xj);
            e = (float)ed;
            sa += (double)__fmul_rn(e, (float)inv);
        }
        out[j] = e;
    }
    float4 r = row[idx];
    r.x = (float)li;
    r.y = (float)(C - sa);
    row[idx] = r;
    Ctab[idx] = (float)C;
}

__global__ void frozen_drift_kernel(const double *lam, const double *x, const double *W,
                                    const double *w0, int n, int Q, double c, double *b0)
{
    __shared__ double red[kMaxQP];
    const int k = blockIdx.x, j = threadIdx.x;
    double P = 1.0, scont = 0.0;
    const double xj = (j < Q) ? x[j] : 0.0;
    const double inv = (j < Q) ? W[j] / (xj * xj) : 0.0;
    for (int i = n; i >= 1; --i) {
        const double li = lam[(size_t)k * n + (i - 1)];
        double contrib = 0.0;
        if (j < Q) {
            const double e = expm1(li * xj);
            contrib = inv * (e * P - li * xj);
            P *= 1.0 + w0[i - 1] * e;
        }
        red[j] = contrib;
        __syncthreads();
        if (j == 0) {
            double A = 0.0;
            for (int t = 0; t < Q; ++t) A += red[t];
            b0[(size_t)k * n + (i - 1)] = -A - 0.5 * c * li * li - c * li * scont;
        }
        scont += w0[i - 1] * li;
        __syncthreads();
    }
}

__global__ void prefix_kernel(const double *b0, int n, int S, double h, float4 *row)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    double D = 0.0;
    for (int k = 0; k < S; ++k) {
        const double bh = b0[(size_t)k * n + l] * h;
        float4 r = row[(size_t)k * n + l];
        r.z = (float)D;
        r.w = (float)bh;
        row[(size_t)k * n + l] = r;
        D += bh;
    }
}

__global__ void finalize_kernel(const double *partials, int grid, int n_out, double *sums)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_out) return;
    double s = 0.0, c = 0.0;
    for (int b = 0; b < grid; ++b) {
        const double y = partials[(size_t)b * n_out + e] - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
    sums[e] = s;
}

// Per instance of a batch: add the partials of its work items in tile order.
__global__ void batch_finalize_kernel(const double *partials, const size_t *seg_off, const int *inst_seg_ptr,
                                      const int *inst_segs, const size_t *out_off, const int *out_count,
                                      double *sums)
{
    const int q = blockIdx.x;
    for (int e = threadIdx.x; e < out_count[q]; e += blockDim.x) {
        double s = 0.0, c = 0.0;
        for (int k = inst_seg_ptr[q]; k < inst_seg_ptr[q + 1]; ++k) {
            const double y = partials[seg_off[inst_segs[k]] + e] - c;
            const double t = s + y;
            c = (t - s) - y;
            s = t;
        }
        sums[out_off[q] + e] = s;
    }
}

}  // namespace

int batch_finalize(const double *partials, const size_t *seg_off, const int *inst_seg_ptr, const int *inst_segs,
                   const size_t *out_off, int n_inst, const int *out_count, double *sums, cudaStream_t st)
{
    batch_finalize_kernel<<<n_inst, 128, 0, st>>>(partials, seg_off, inst_seg_ptr, inst_segs, out_off, out_count,
                                                  sums);
    return (int)cudaGetLastError();
}

int launch_tables(const double *lam, const double *x, const double *W, int n, int S, int Q, int QP,
                  float4 *tab, float *cn, float4 *row, float *Ctab, cudaStream_t st)
{
    const int total = S * n;
    tables_kernel<<<(total + 127) / 128, 128, 0, st>>>(lam, x, W, n, S, Q, QP, tab, cn, row, Ctab);
    return (int)cudaGetLastError();
}

int launch_frozen_drift(const double *lam, const double *x, const double *W, const double *w0,
                        int n, int S, int Q, double c, double h, double *b0, float4 *row,
                        cudaStream_t st)
{
    frozen_drift_kernel<<<S, kMaxQP, 0, st>>>(lam, x, W, w0, n, Q, c, b0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    prefix_kernel<<<(n + 127) / 128, 128, 0, st>>>(b0, n, S, h, row);
    return (int)cudaGetLastError();
}

int launch_finalize(const double *partials, int grid, int n_out, double *sums, cudaStream_t st)
{
    finalize_kernel<<<(n_out + 127) / 128, 128, 0, st>>>(partials, grid, n_out, sums);
    return (int)cudaGetLastError();
}

}  // namespace lll
