// lll_mlp.cu -- the learned compensator: BF16 tensor-core training and
// inference kernels of a small SiLU MLP (FP32 accumulation, FP32 master
// weights, Adam).
//
// The network stands in for the jump-compensator integral of
// Eq. (LIBOR-drift-PT) in the full scheme.  It maps a feature row
//   (t / T_N, i / n, lambda(t, T_i) / lambda_ref, u_0 .. u_{N-1}),
//   u_m = (log L_m(t) - log L_m(0)) * u_scale,
// to y = (A_i - C_i) / y_scale, the state-dependent part of the compensator in
// scaled units (C_i, the compensator at zero weights, is exact and cheap, so
// the network only has to learn the part that depends on the later rates).
//
// Kernels:
//   gemm_bf16        C = op(A) op(B) with mma.sync.m16n8k16 (BF16 in, FP32
//                    accumulate), optional split-K partials, fused epilogues
//                    (bias + SiLU for the forward pass, SiLU' for the backward).
//   out_loss         output layer (dot product), residual, MSE loss partials.
//   reduce_*         deterministic fixed-order reductions (split-K, bias grads).
//   adam             Adam on FP32 master weights, BF16 copies for the GEMMs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lll_internal.h"
#include "lll_mlp.h"

namespace lll {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// SiLU(z) = z sigma(z) with sigma(z) = (1 + tanh(z/2)) / 2 (one MUFU op); the
// fused inference kernel uses the same form.
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu(float z) { return 0.5f * z * (1.0f + tanh_approx(0.5f * z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 0.5f * (1.0f + tanh_approx(0.5f * z));
    return s * (1.0f + z * (1.0f - s));
}

// C[M x N] = sum_k A(m, k) B(k, n) over the K range of blockIdx.z.
//   A(m, k) = A[m * lda + k]  (TA = 0)   or  A[k * lda + m]  (TA = 1)
//   B(k, n) = B[k * ldb + n]  (TB = 0)   or  B[n * ldb + k]  (TB = 1)
// EPI 0: write FP32 C (+ z * M * N for split-K partials).
// EPI 1: z = C + bias[n]; Zout = z (FP32, if given); Hout = bf16(SiLU(z)).
// EPI 2: Hout = bf16(C * SiLU'(Zin[m, n])); Zout = that value in FP32.
template <int TA, int TB, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16(const __nv_bfloat16 *__restrict__ A, int lda,
                                                 const __nv_bfloat16 *__restrict__ B, int ldb,
                                                 int M, int N, int K, int k_chunk, float *C,
                                                 const float *bias, const float *Zin, float *Zout,
                                                 __nv_bfloat16 *Hout)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * k_chunk, ke = min(K, kb + k_chunk);
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 128) {
            const int mm = TA ? (e % BM) : (e / BK), kk = TA ? (e / BM) : (e % BK);
            const int gm = m0 + mm, gk = k0 + kk;
            __nv_bfloat16 v = zero;
            if (gm < M && gk < ke) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[mm][kk] = v;
        }
        for (int e = tid; e < BN * BK; e += 128) {
            const int nn = TB ? (e / BK) : (e % BN), kk = TB ? (e % BK) : (e / BN);
            const int gn = n0 + nn, gk = k0 + kk;
            __nv_bfloat16 v = zero;
            if (gn < N && gk < ke) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[nn][kk] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            const int r = lane >> 2, c = (lane & 3) * 2;
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int row = wm + mt * 16 + r;
                af[mt][0] = *reinterpret_cast<const uint32_t *>(&As[row][ks + c]);
                af[mt][1] = *reinterpret_cast<const uint32_t *>(&As[row + 8][ks + c]);
                af[mt][2] = *reinterpret_cast<const uint32_t *>(&As[row][ks + c + 8]);
                af[mt][3] = *reinterpret_cast<const uint32_t *>(&As[row + 8][ks + c + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int col = wn + nt * 8 + r;
                bf[nt][0] = *reinterpret_cast<const uint32_t *>(&Bs[col][ks + c]);
                bf[nt][1] = *reinterpret_cast<const uint32_t *>(&Bs[col][ks + c + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
        }
        __syncthreads();
    }
    // C fragment: rows r and r + 8, columns c, c + 1 of each 16 x 8 tile.
    const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int gm = m0 + wm + mt * 16 + r + ((h >> 1) << 3);
                const int gn = n0 + wn + nt * 8 + c + (h & 1);
                if (gm >= M || gn >= N) continue;
                const float v = acc[mt][nt][h];
                const size_t o = (size_t)gm * N + gn;
                if (EPI == 0) {
                    C[(size_t)blockIdx.z * M * N + o] = v;
                } else if (EPI == 1) {
                    const float z = v + bias[gn];
                    if (Zout) Zout[o] = z;
                    Hout[o] = __float2bfloat16(silu(z));
                } else {
                    const float d = v * silu_grad(Zin[o]);
                    Zout[o] = d;
                    Hout[o] = __float2bfloat16(d);
                }
            }
}

// Output layer, residual and loss: out[r] = H[r] . w + b; d[r] = 2 (out - y) / rows
// (dL/dout); per-block loss partials.  One warp per row.
__global__ void out_loss(const __nv_bfloat16 *H, int Hdim, const __nv_bfloat16 *w, const float *b,
                         const float *y, int rows, float *out, float *dout, double *loss_part)
{
    __shared__ double red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + warp;
    double l = 0.0;
    if (row < rows) {
        float s = 0.0f;
        for (int c = lane; c < Hdim; c += 32)
            s += __bfloat162float(H[(size_t)row * Hdim + c]) * __bfloat162float(w[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        s += b[0];
        if (lane == 0) {
            out[row] = s;
            if (y) {
                const float rr = s - y[row];
                dout[row] = 2.0f * rr / (float)rows;
                l = (double)rr * rr;
            }
        }
    }
    if (lane == 0) red[warp] = l;
    __syncthreads();
    if (threadIdx.x == 0 && loss_part) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += red[i];
        loss_part[blockIdx.x] = t;
    }
}

// Vector head: out[r, o] += b[o] for o < O (out from the output GEMM); with
// targets y (rows x O) and the rows' Euler steps kr, the masked residual
// over the live rates (o + 1 >= kr / s + 1, o < n): dout = 2 (out - y) / (rows n)
// (FP32 and BF16), per-block sums of squares and live counts.  One thread per
// element (consecutive threads, consecutive outputs of a row: coalesced);
// blocks of 128 elements, so the per-block partials are in a fixed order.
__global__ void vec_loss(float *out, const float *b, const float *y, const int *kr, int rows, int O, int n, int s,
                         float *dout, __nv_bfloat16 *douth, double *loss_part, double *cnt_part)
{
    __shared__ double red[2][128];
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0, c = 0.0;
    if (e < (size_t)rows * O) {
        const int r = (int)(e / O), o = (int)(e % O);
        const float v = out[e] + b[o];
        out[e] = v;
        if (y) {
            const int imin = kr[r] / s + 1;
            float d = 0.0f;
            if (o < n && o + 1 >= imin) {
                const float rr = v - y[e];
                d = 2.0f / ((float)rows * (float)n) * rr;
                l = (double)rr * rr;
                c = 1.0;
            }
            dout[e] = d;
            douth[e] = __float2bfloat16(d);
        }
    }
    red[0][threadIdx.x] = l;
    red[1][threadIdx.x] = c;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            red[0][threadIdx.x] += red[0][threadIdx.x + k];
            red[1][threadIdx.x] += red[1][threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_part) {
        loss_part[blockIdx.x] = red[0][0];
        cnt_part[blockIdx.x] = red[1][0];
    }
}

// dZ_L[r, c] = dout[r] * w[c] * SiLU'(Z_L[r, c]), FP32 and BF16 copies.
__global__ void out_backward(const float *dout, const __nv_bfloat16 *w, const float *Z, int rows,
                             int Hdim, float *dZ, __nv_bfloat16 *dZh)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)rows * Hdim) return;
    const int r = (int)(e / Hdim), c = (int)(e % Hdim);
    const float d = dout[r] * __bfloat162float(w[c]) * silu_grad(Z[e]);
    dZ[e] = d;
    dZh[e] = __float2bfloat16(d);
}

// Column sums in two fixed-order passes (bias and output-weight gradients):
// pass 1, block (32-column group, chunk of kColRows rows), 32 x 8 threads:
// thread (c, y) adds rows y, y + 8, .. of the chunk in column c (a warp reads
// 32 consecutive columns of a row: coalesced), then the 8 row-lanes are added
// in order into part[chunk][c]; pass 2 adds the chunks in order.  With a row
// weight w the sums are sum_r w[r] X[r, c], and column `cols` (one past the
// last) is sum_r w[r] (the bias of the output layer).
constexpr int kColRows = 256;

template <typename T>
__global__ void __launch_bounds__(256) colsum_part(const T *X, const float *w, int rows, int cols, int with_ones,
                                                   float *part)
{
    __shared__ float red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int width = cols + with_ones;
    const int r0 = blockIdx.y * kColRows, r1 = min(rows, r0 + kColRows);
    float s = 0.0f;
    if (c < width) {
        for (int r = r0 + ty; r < r1; r += 8) {
            const float x = c < cols ? (float)X[(size_t)r * cols + c] : 1.0f;
            s += w ? w[r] * x : x;
        }
    }
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && c < width) {
        float t = red[0][tx];
        for (int y = 1; y < 8; ++y) t += red[y][tx];
        part[(size_t)blockIdx.y * width + c] = t;
    }
}

__global__ void colsum_final(const float *part, int chunks, int width, float *out, float *out_extra)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= width) return;
    float s = 0.0f;
    for (int z = 0; z < chunks; ++z) s += part[(size_t)z * width + c];
    if (out_extra && c == width - 1) out_extra[0] = s;
    else out[c] = s;
}

// Transposed BF16 copies of weight matrices: dst[off + c rows + r] = src[off + r cols + c].
struct TransposeJobs {
    size_t off[6];
    int rows[6], cols[6];
    int count;
};

__global__ void transpose_bf16(const __nv_bfloat16 *src, __nv_bfloat16 *dst, TransposeJobs jobs)
{
    const int j = blockIdx.y;
    if (j >= jobs.count) return;
    const int rows = jobs.rows[j], cols = jobs.cols[j];
    const size_t off = jobs.off[j];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)rows * cols; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        dst[off + (size_t)c * rows + r] = src[off + e];
    }
}

// Sum of split-K partials in a fixed order: four running sums over the splits
// z = 0, 4, 8, .. / 1, 5, .. / 2, .. / 3, .. (independent loads in flight),
// then added as ((s0 + s1) + (s2 + s3)).
__global__ void reduce_splits(const float *part, int splits, size_t count, float *out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int z = 0;
    for (; z + 4 <= splits; z += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] += part[(size_t)(z + u) * count + e];
    }
    for (int u = 0; z < splits; ++z, ++u) s[u] += part[(size_t)z * count + e];
    out[e] = (s[0] + s[1]) + (s[2] + s[3]);
}

__global__ void adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *ph, size_t count,
                     float lr, float b1, float b2, float eps, float c1, float c2)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float upd = lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    const float np = p[e] - upd;
    p[e] = np;
    if (ph) ph[e] = __float2bfloat16(np);
}

__global__ void to_bf16(const float *x, size_t count, __nv_bfloat16 *y)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) y[e] = __float2bfloat16(x[e]);
}

unsigned blocks_for(size_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------------------
// Host-side launch helpers (used by lll_mlp_host.cpp).
// ---------------------------------------------------------------------------
int mlp_gemm_mma(int ta, int tb, int epi, const void *A, int lda, const void *B, int ldb, int M, int N,
                 int K, int splits, float *C, const float *bias, const float *Zin, float *Zout, void *Hout,
                 cudaStream_t st)
{
    if (splits < 1) splits = 1;
    int k_chunk = (K + splits - 1) / splits;
    k_chunk = ((k_chunk + BK - 1) / BK) * BK;
    splits = (K + k_chunk - 1) / k_chunk;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    const auto *a = static_cast<const __nv_bfloat16 *>(A);
    const auto *b = static_cast<const __nv_bfloat16 *>(B);
    auto *h = static_cast<__nv_bfloat16 *>(Hout);
#define LLL_GEMM(TA_, TB_, EPI_)                                                                   \
    gemm_bf16<TA_, TB_, EPI_><<<grid, 128, 0, st>>>(a, lda, b, ldb, M, N, K, k_chunk, C, bias, Zin, \
                                                   Zout, h)
    if (epi == 0 && ta == 0 && tb == 0) LLL_GEMM(0, 0, 0);
    else if (epi == 0 && ta == 1 && tb == 0) LLL_GEMM(1, 0, 0);
    else if (epi == 0 && ta == 0 && tb == 1) LLL_GEMM(0, 1, 0);
    else if (epi == 1 && ta == 0 && tb == 1) LLL_GEMM(0, 1, 1);
    else if (epi == 2 && ta == 0 && tb == 0) LLL_GEMM(0, 0, 2);
    else return (int)cudaErrorInvalidValue;
#undef LLL_GEMM
    return (int)cudaGetLastError();
}

int mlp_splits_used_mma(int K, int splits)
{
    if (splits < 1) splits = 1;
    int k_chunk = (K + splits - 1) / splits;
    k_chunk = ((k_chunk + BK - 1) / BK) * BK;
    return (K + k_chunk - 1) / k_chunk;
}

int mlp_out_loss(const void *H, int Hdim, const void *w, const float *b, const float *y, int rows,
                 float *out, float *dout, double *loss_part, cudaStream_t st)
{
    out_loss<<<(rows + 7) / 8, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(H), Hdim,
                                            static_cast<const __nv_bfloat16 *>(w), b, y, rows, out,
                                            dout, loss_part);
    return (int)cudaGetLastError();
}

int mlp_vec_loss(float *out, const float *b, const float *y, const int *kr, int rows, int O, int n, int s,
                 float *dout, void *douth, double *loss_part, double *cnt_part, cudaStream_t st)
{
    const size_t count = (size_t)rows * O;
    vec_loss<<<blocks_for(count, 128), 128, 0, st>>>(out, b, y, kr, rows, O, n, s, dout,
                                                     static_cast<__nv_bfloat16 *>(douth), loss_part, cnt_part);
    return (int)cudaGetLastError();
}

int mlp_out_backward(const float *dout, const void *w, const float *Z, int rows, int Hdim, float *dZ,
                     void *dZh, cudaStream_t st)
{
    const size_t count = (size_t)rows * Hdim;
    out_backward<<<blocks_for(count, 256), 256, 0, st>>>(dout, static_cast<const __nv_bfloat16 *>(w),
                                                         Z, rows, Hdim, dZ,
                                                         static_cast<__nv_bfloat16 *>(dZh));
    return (int)cudaGetLastError();
}

int mlp_colsum_chunks(int rows) { return (rows + kColRows - 1) / kColRows; }

int mlp_out_weight_grad(const float *dout, const void *H, int rows, int Hdim, float *gw, float *gb, float *part,
                        cudaStream_t st)
{
    const int width = Hdim + 1, chunks = mlp_colsum_chunks(rows);
    colsum_part<__nv_bfloat16><<<dim3((width + 31) / 32, chunks), 256, 0, st>>>(
        static_cast<const __nv_bfloat16 *>(H), dout, rows, Hdim, 1, part);
    colsum_final<<<(width + 127) / 128, 128, 0, st>>>(part, chunks, width, gw, gb);
    return (int)cudaGetLastError();
}

int mlp_column_sums(const float *X, int rows, int cols, float *out, float *part, cudaStream_t st)
{
    const int chunks = mlp_colsum_chunks(rows);
    colsum_part<float><<<dim3((cols + 31) / 32, chunks), 256, 0, st>>>(X, nullptr, rows, cols, 0, part);
    colsum_final<<<(cols + 127) / 128, 128, 0, st>>>(part, chunks, cols, out, nullptr);
    return (int)cudaGetLastError();
}

int mlp_transpose_weights(const void *src, void *dst, const size_t *off, const int *rows, const int *cols, int count,
                          cudaStream_t st)
{
    if (count < 1 || count > 6) return (int)cudaErrorInvalidValue;
    TransposeJobs jobs{};
    for (int j = 0; j < count; ++j) {
        jobs.off[j] = off[j];
        jobs.rows[j] = rows[j];
        jobs.cols[j] = cols[j];
    }
    jobs.count = count;
    transpose_bf16<<<dim3(64, count), 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(src),
                                                    static_cast<__nv_bfloat16 *>(dst), jobs);
    return (int)cudaGetLastError();
}

int mlp_reduce_splits(const float *part, int splits, size_t count, float *out, cudaStream_t st)
{
    reduce_splits<<<blocks_for(count, 256), 256, 0, st>>>(part, splits, count, out);
    return (int)cudaGetLastError();
}

int mlp_adam(float *p, const float *g, float *m, float *v, void *ph, size_t count, float lr, float b1,
             float b2, float eps, int t, cudaStream_t st)
{
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam<<<blocks_for(count, 256), 256, 0, st>>>(p, g, m, v, static_cast<__nv_bfloat16 *>(ph), count,
                                                 lr, b1, b2, eps, c1, c2);
    return (int)cudaGetLastError();
}

int mlp_to_bf16(const float *x, size_t count, void *y, cudaStream_t st)
{
    to_bf16<<<blocks_for(count, 256), 256, 0, st>>>(x, count, static_cast<__nv_bfloat16 *>(y));
    return (int)cudaGetLastError();
}

}  // namespace lll
