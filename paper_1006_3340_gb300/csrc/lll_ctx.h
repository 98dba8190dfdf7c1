// lll_ctx.h -- the model context behind the opaque lll_ctx handle (private).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lll.h"

namespace lll {
struct MlpState;
void mlp_free(MlpState *m);
}  // namespace lll

struct lll_ctx {
    int N = 0, n = 0, s = 0, S = 0, Q = 0, QP = 0, driver = 0;
    double delta = 0, h = 0, c = 0, mu = 0, gam = 0, BN = 0;
    lll_nig nig{};
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    std::vector<double> L0;
    // device
    double *d_lam = nullptr, *d_x = nullptr, *d_W = nullptr, *d_w0 = nullptr, *d_b0 = nullptr;
    float4 *d_tab = nullptr, *d_row = nullptr;
    float *d_cn = nullptr; // [QP]: c_j = W_j / x_j^2
    float *d_C = nullptr; // [S][n]: C_l(t_k), the compensator at zero weights (FP64-built)
    float *d_Z0 = nullptr, *d_c0 = nullptr, *d_strikes = nullptr;
    double *d_partials = nullptr, *d_sums = nullptr;
    size_t partials_cap = 0, sums_cap = 0;
    float *d_state = nullptr;
    size_t state_cap = 0;
    float *d_snap = nullptr;
    uint64_t n_snap = 0, snap_stride = 1;
    int ns = 0;
    int product = 0; // LLL_PRODUCT_*
    bool simulated = false;
    uint64_t last_paths = 0;
    uint64_t last_snap_paths = 0;
    int threads = 128, blocks_per_sm = 0, chunk_rows = 0, ppt = 0, lpp = 0; // 0: automatic
    int tenor_lanes = 0; // > 0: full and Picard on the tenor-parallel kernel (lll_set_mapping)
    bool step_map = false; // Picard with its Euler steps in parallel (lll_set_mapping)
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::vector<double> lam; // host copy of lambda [S][n]
    lll::MlpState *mlp = nullptr;
    int mlp_kernel = 0;     // LLL_MLP_KERNEL_*
    float *d_K1 = nullptr, *d_K2 = nullptr, *d_K3 = nullptr; // drift-expansion tables
    int expand_order = 0;   // order the tables were built for (0: none)
    int *d_err = nullptr;   // error word of kernels with bounded waits
    int inject = 0;         // LLL_INJECT_* for the next launch (failure-detection tests)
    bool err_pending = false;
    bool gemm_err_pending = false; // the last simulation ran the layered GEMMs (their error word)
    std::string err;
};
