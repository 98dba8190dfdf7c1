// lll_mlp.h -- launch helpers of the MLP kernels (lll_mlp.cu, lll_mlp_path.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lll_internal.h"

namespace lll {

// Split-K aware BF16 GEMM (see lll_mlp.cu for the operand conventions): the
// tcgen05 kernel (lll_gemm_tc.cu, the default) or the mma.sync kernel
// (lll_mlp.cu), chosen process-wide by lll_set_gemm_kernel.
int mlp_gemm(int ta, int tb, int epi, const void *A, int lda, const void *B, int ldb, int M, int N,
             int K, int splits, float *C, const float *bias, const float *Zin, float *Zout, void *Hout,
             cudaStream_t st);
int mlp_splits_used(int K, int splits);
int mlp_gemm_kind(); // LLL_GEMM_TC or LLL_GEMM_MMA_SYNC (epilogue 3, C + bias, is tcgen05 only)
int mlp_gemm_mma(int ta, int tb, int epi, const void *A, int lda, const void *B, int ldb, int M, int N,
                 int K, int splits, float *C, const float *bias, const float *Zin, float *Zout, void *Hout,
                 cudaStream_t st);
int mlp_splits_used_mma(int K, int splits);
int mlp_gemm_tc(int ta, int tb, int epi, const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                int splits, float *C, const float *bias, const float *Zin, float *Zout, void *Hout, int *err,
                cudaStream_t st);
int mlp_splits_used_tc(int K, int splits);
// lll_gemm_tc.cu: a TMA tensor map (declared as void storage of 128 bytes, the
// size of a CUtensorMap) of a row-major BF16 matrix [rows x K], leading
// dimension ld (a multiple of 8), boxes {64, box_rows}, 128-byte swizzle.
bool make_tmap(struct CUtensorMap_st *tm, const void *base, int rows, int K, int ld, int box_rows);

int mlp_out_loss(const void *H, int Hdim, const void *w, const float *b, const float *y, int rows,
                 float *out, float *dout, double *loss_part, cudaStream_t st);
int mlp_vec_loss(float *out, const float *b, const float *y, const int *kr, int rows, int O, int n, int s,
                 float *dout, void *douth, double *loss_part, double *cnt_part, cudaStream_t st);
int mlp_out_backward(const float *dout, const void *w, const float *Z, int rows, int Hdim, float *dZ,
                     void *dZh, cudaStream_t st);
// Column sums in two fixed-order passes through part[mlp_colsum_chunks(rows)][cols + 1].
int mlp_colsum_chunks(int rows);
int mlp_out_weight_grad(const float *dout, const void *H, int rows, int Hdim, float *gw, float *gb, float *part,
                        cudaStream_t st);
int mlp_column_sums(const float *X, int rows, int cols, float *out, float *part, cudaStream_t st);
// BF16 transposes of up to six weight matrices at the same flat offsets: dst
// holds [cols][rows] where src holds [rows][cols].
int mlp_transpose_weights(const void *src, void *dst, const size_t *off, const int *rows, const int *cols, int count,
                          cudaStream_t st);
int mlp_reduce_splits(const float *part, int splits, size_t count, float *out, cudaStream_t st);
int mlp_adam(float *p, const float *g, float *m, float *v, void *ph, size_t count, float lr, float b1,
             float b2, float eps, int t, cudaStream_t st);
int mlp_to_bf16(const float *x, size_t count, void *y, cudaStream_t st);

// Feature scaling of the network input row (see lll_mlp.cu).
struct MlpScales {
    float t_scale;      // 1 / T_N
    float i_scale;      // 1 / n
    float lam_scale;    // 1 / lambda_ref
    float u_scale;      // multiplier of log L_m(t) - log L_m(0)
    float y_scale;      // target unit: A_i - C_i = y_scale * f(x)
};

// Network arguments of the fused LLL_MLP path kernel.
struct MlpArgs {
    const __nv_bfloat16 *wh; // BF16 copy of the flat parameters
    const float *wp;         // FP32 flat parameters (biases are read from here)
    size_t offW[4], offb[4], off_wout, off_bout;
    MlpScales sc;
    const float *Ctab;       // [S][n] compensator at zero weights
    int in_pad;              // padded input width of layer 0
    int *err;                // tensor-core kernel: set non-zero when a wait timed out
    int stall_mma;           // failure-detection test: the MMA warp issues nothing
};

// lll_mlp_path.cu
int mlp_path_threads();
size_t mlp_path_smem(int layers, int in_pad, int n, int ns);
bool mlp_path_supported(int hidden, int layers, int in_pad);
int mlp_path_occupancy(int layers, int in_pad, size_t smem, int *blocks_per_sm);
int launch_mlp_path(int layers, int in_pad, int grid, size_t smem, cudaStream_t st, const PathArgs &a,
                    const MlpArgs &g);

// lll_mlp_layered.cu (any network: layer-by-layer over the rows of a step)
int mlp_layered_threads();
int launch_mlp_features(const PathArgs &a, const MlpScales &sc, int k, int Pc, const float *state, void *X,
                        int in_pad, int head, cudaStream_t st);
// out_t: the vector head's outputs are [outputs][Pc] (rates as rows), else [Pc][outputs]
int launch_mlp_euler(const PathArgs &a, const float *Ctab, float y_scale, int k, uint64_t chunk_first, int Pc,
                     float *state, const float *out, int outputs, int out_t, double *acc, cudaStream_t st);
int launch_mlp_acc_to_partials(const double *acc, size_t cells, double *partials, cudaStream_t st);

// lll_mlp_tc.cu (tcgen05, accumulators in tensor memory; hidden = 128)
int mlp_tc_threads();
int mlp_tc_paths_per_block();
size_t mlp_tc_smem(int layers, int in_pad, int n, int ns);
bool mlp_tc_supported(int hidden, int layers, int in_pad);
int mlp_tc_occupancy(int layers, int in_pad, size_t smem, int *blocks_per_sm);
int launch_mlp_tc(int layers, int in_pad, int grid, size_t smem, cudaStream_t st, const PathArgs &a,
                  const MlpArgs &g);
// vector head (one pass per path and step, 48 output columns)
size_t mlp_tc_vec_smem(int layers, int in_pad, int n, int ns);
bool mlp_tc_vec_supported(int hidden, int layers, int in_pad, int outputs, int n);
int mlp_tc_vec_occupancy(int layers, int in_pad, size_t smem, int *blocks_per_sm);
int launch_mlp_tc_vec(int layers, int in_pad, int grid, size_t smem, cudaStream_t st, const PathArgs &a,
                      const MlpArgs &g);

// lll_mlp_wide.cu (tcgen05, vector head of width 256: the whole simulation in
// one persistent kernel, one 128-path tile per CTA at a time, weights streamed
// by TMA; acc: [grid][n][ns][4] FP64 Kahan sums, zeroed by the caller)
size_t mlp_wide_smem(int n, int ns);
bool mlp_wide_supported(int hidden, int layers, int in_pad, int outputs, int n, int ns, int product);
int launch_mlp_wide(int layers, int in_pad, int outputs, int grid, cudaStream_t st, const PathArgs &a,
                    const MlpArgs &g, double *acc);

}  // namespace lll
