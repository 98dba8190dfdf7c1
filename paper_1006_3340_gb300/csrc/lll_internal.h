// lll_internal.h -- structures shared by the translation units of liblll.so.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lll {

enum Scheme { FULL = 0, PICARD = 1, MLP = 2, FROZEN = 3, EXPAND1 = 4, EXPAND2 = 5 };

// Largest padded node count the path kernels are compiled for.
constexpr int kMaxQP = 128;
// Maximum threads per block of the path kernels.
constexpr int kMaxThreads = 256;

// Arguments of the path kernels (one simulation of one scheme).
struct PathArgs {
    const float4 *tab;    // [S][n][QP/4]: (E_j .. E_j+3), E_lj = e^{lambda_l(t_k) x_j} - 1
    const float *cn;      // [QP]: c_j = W_j / x_j^2 (0 on padding nodes)
    const float4 *row;    // [S][n]: (lambda_l(t_k), K_l(k), D0_l(t_k), b0_l(t_k) * h)
    const float *Z0;      // [n]: log L(0, T_l)
    const float *c0;      // [n]: log L(0, T_l) + log delta
    const float *strikes; // [n][ns]
    double *partials;     // [grid][n][ns][2]: per-block payoff sum and sum of squares
    float *state;         // [grid][nst][n][threads]: per-path state (log-rate offsets)
    float *snap;          // [n][n][n_snap]: log L_l(T_m) for the first n_snap paths, or null
    uint64_t n_snap, snap_stride, snap_pitch; // recorded paths, path stride, row pitch of snap
    uint64_t first_path, paths;
    int n, s, S, ns, chunk_rows;
    uint32_t key0, key1, inst;
    int driver;           // 0 NIG, 1 Brownian
    float h, sqrt_h, delta, dBN; // dBN = delta * B(0, T_N)
    int product;          // 0: caplets, 1: co-terminal payer swaptions (see lll_device.cuh)
    // NIG increment over one step: IG(mean m, shape l) mixing variable.
    float ig_m, ig_m2, ig_hl, ig_fl; // m, m^2, m / (2 l), 4 m l
    float nig_beta, nig_muh;         // beta, mu * h
    double ig_md, ig_ld;             // m and l in FP64 for the acceptance re-check
};

// Many instances in one persistent launch (see batch_kernel in lll_paths.cu).
struct BatchArgs {
    const PathArgs *desc;    // [n_inst] per-instance arguments (state/partials unused)
    const int *item_inst;    // [items] instance of each work item (items in claiming order)
    const uint2 *item_tiles; // [items] tile range [x, y) of the item within its instance
    const size_t *seg_off;   // [items] offset (doubles) of each item's output in partials
    double *partials;        // item outputs: [n][ns][2] per item
    float *state;            // [grid][NST][n_max][threads]
    int *next;               // claim counter, 0 at launch
    int n_items, n_max, ns_max, chunk_rows;
};

// The launch lll_simulate would make for one simulation, worked out without
// allocating anything; state and partials are left for the caller to place.
struct LaunchPlan {
    PathArgs args;
    int scheme, qp, ppt, lpp, threads, grid; // lpp: lanes per group of paths (1, 2 or 4)
    int tenor;                               // > 0: tenor-parallel kernel with this many lanes per path
    size_t smem;
    size_t state_floats_per_block, partial_doubles_per_block;
    int n_out; // doubles written by the final reduction: n * n_strikes * 2
    cudaStream_t stream;
    int device;
};

// Launchers implemented in lll_paths.cu.  Return a cudaError_t value.
// R = paths carried per thread (1, or 2 where compiled: padded Q <= 64).
int launch_path_kernel(int scheme, int QP, int R, int grid, int threads, size_t smem, cudaStream_t st,
                       const PathArgs &a);
int path_kernel_occupancy(int scheme, int QP, int R, int threads, size_t smem, int *blocks_per_sm);
int path_kernel_prepare(int scheme, int QP, int R, int threads, size_t smem);
bool path_kernel_supported(int scheme, int QP, int R);
size_t path_kernel_smem(int QP, int n, int ns, int threads, int chunk_rows);

// Launchers implemented in lll_paths_group.cu (four lanes per group of four paths).
bool group_kernel_supported(int scheme, int QP, int G);
size_t group_kernel_smem(int QP, int n, int ns, int threads, int chunk_rows);
int group_kernel_prepare(int scheme, int QP, int G, size_t smem, int threads, int *blocks_per_sm);
int launch_group_kernel(int scheme, int QP, int G, int grid, int threads, size_t smem, cudaStream_t st,
                        const PathArgs &a);
// Launchers implemented in lll_paths_tenor.cu (G lanes per path, each owning a block of rates).
int tenor_rates_per_lane(int n, int G);
bool tenor_kernel_supported(int scheme, int QP, int G);
size_t tenor_kernel_smem(int QP, int n, int ns, int G);
int tenor_kernel_threads();
int tenor_kernel_prepare(int scheme, int QP, int G, size_t smem, int *blocks_per_sm);
int launch_tenor_kernel(int scheme, int QP, int G, int grid, size_t smem, cudaStream_t st, const PathArgs &a);
// Launchers implemented in lll_paths_step.cu (Picard with its Euler steps in parallel).
bool step_kernels_supported(int QP, int ns);
size_t step_bytes_per_path(int n, int S);
int step_blocks_per_chunk(int Pc);
int launch_step_chunk(int QP, const PathArgs &a, uint64_t chunk_first, int Pc, float *dH, float *Y, float *Bh,
                      float *Zm, int block0, double *partials, cudaStream_t st);
struct LaunchPlan;
int launch_plan(const LaunchPlan &plan, const PathArgs &a);
bool batch_kernel_supported(int scheme, int QP, int R);
int batch_kernel_prepare(int scheme, int QP, int R, size_t smem, int threads, int *blocks_per_sm);
int launch_batch_kernel(int scheme, int QP, int R, int grid, int threads, size_t smem, cudaStream_t st,
                        const BatchArgs &b);

// Launchers implemented in lll_tables.cu.
int launch_tables(const double *lam, const double *x, const double *W, int n, int S, int Q, int QP,
                  float4 *tab, float *cn, float4 *row, float *Ctab, cudaStream_t st);
int launch_frozen_drift(const double *lam, const double *x, const double *W, const double *w0,
                        int n, int S, int Q, double c, double h, double *b0, float4 *row,
                        cudaStream_t st);
int launch_finalize(const double *partials, int grid, int n_out, double *sums, cudaStream_t st);

// Implemented in lll_gemm_tc.cu: read and clear the error word of the tcgen05
// GEMMs on the current device (non-zero: a bounded wait gave up since the
// last read).  Synchronises the stream.
int mlp_gemm_take_error(int *word, cudaStream_t st);

}  // namespace lll

struct lll_ctx;
namespace lll {
// Implemented in lll_capi.cpp.
// allow_tenor: honour the context's tenor-parallel mapping (lll_set_mapping);
// callers that only need the path arguments of the full scheme pass false.
int plan_launch(lll_ctx *ctx, int scheme, uint64_t first_path, uint64_t paths, uint64_t seed,
                LaunchPlan *plan, bool allow_tenor = true);
int record_error(lll_ctx *ctx, int code, const char *msg);
}  // namespace lll
