/*
 * lll.h -- C ABI of liblll.so: GB300 (sm_103a) Monte Carlo of the Levy LIBOR
 * model under the terminal measure, after A. Papapantoleon and D. Skovmand,
 * "Numerical Methods for the Levy LIBOR model" (arXiv 1006.3340).
 *
 * Conventions used by every call
 * ------------------------------
 *  - Tenor (Section 2): accrual dates T_k = k * delta, k = 0..N, terminal
 *    date T_N = T_*.  The simulated rates are L_m = L(., T_m), m = 1..n with
 *    n = N - 1 (the paper's N); L_0 is the spot rate, known at t = 0.
 *  - Time grid: s Euler steps per accrual period, h = delta / s, t_k = k h,
 *    k = 0..n*s-1.  Rate i is simulated while k < i*s (it fixes at T_i).
 *  - All host arrays are row-major, owned by the caller, read during the
 *    call only (inputs are copied into library-owned device memory).
 *  - Every device buffer is allocated and owned by the library and is freed
 *    by lll_destroy.  Work is issued on the stream given to lll_init (NULL =
 *    the legacy default stream); calls returning host data synchronise it.
 *  - Every function returns LLL_OK (0) or a negative status.  After an
 *    error, lll_last_error(ctx) gives a message.  LLL_EDOMAIN from lll_init is
 *    a warning: the context is created and usable.
 */
#ifndef LLL_H
#define LLL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LLL_OK 0
#define LLL_EINVAL (-1)      /* null pointer, bad size, NaN/Inf, L0 <= 0, delta <= 0, zero node */
#define LLL_EDOMAIN (-2)     /* NIG sum |lambda| >= alpha - |beta| (LR1 fails for the untruncated
                                measure; the compensator is truncated to the rule's range) */
#define LLL_ECUDA (-3)       /* a CUDA runtime call failed; the message names it */
#define LLL_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define LLL_ENOMEM (-5)      /* device or host allocation failed */
#define LLL_ESTATE (-6)      /* call out of order (e.g. pricing before simulating) */
#define LLL_EUNSUPPORTED (-7)/* size beyond what the compiled kernels handle (Q > 128) */

/* Schemes.  LLL_FULL: the log-Euler scheme of Eq. (log-LIB-SDE-2) with the
 * drift of Eq. (LIBOR-drift-PT) evaluated at the simulated later rates.
 * LLL_PICARD: the drift of Eq. (bdrift), evaluated at the Picard iterate
 * Z^(1) of Eq. (Picard-2) (Section 3.1).  LLL_FROZEN: L^0 = exp(Z^(1)), the
 * frozen-drift approximation (Section 1, Section 3.2).  LLL_MLP: the full
 * scheme with the jump compensator replaced by a trained network.
 * LLL_EXPAND1 / LLL_EXPAND2: the full scheme with the compensator replaced by
 * its first / second order drift expansion, Eq. (drifta) / Eq. (drifta2)
 * (Section 3.3), written with the NIG jump cumulant in closed form (no
 * nodes); NIG driver only, n <= 64 resp. n <= 16 rates (LLL_EUNSUPPORTED
 * beyond), LLL_EDOMAIN if a needed cumulant argument leaves |beta + u| < alpha. */
typedef enum {
    LLL_FULL = 0,
    LLL_PICARD = 1,
    LLL_MLP = 2,
    LLL_FROZEN = 3,
    LLL_EXPAND1 = 4,
    LLL_EXPAND2 = 5
} lll_scheme;

/* Driver H (Section 2, Eq. (canon-LIBOR)).  LLL_DRIVER_NIG: pure-jump NIG
 * (Section 4), drawn as beta V + sqrt(V) Z + mu h with V inverse Gaussian.
 * LLL_DRIVER_BROWNIAN: H = W (c = 1, no jumps), the log-normal LIBOR model. */
typedef enum { LLL_DRIVER_NIG = 0, LLL_DRIVER_BROWNIAN = 1 } lll_driver;

/* NIG parameters (alpha, beta, delta-bar, mu) of H_1.  mu = NaN selects the
 * martingale value -delta_bar * beta / sqrt(alpha^2 - beta^2), which makes H a
 * martingale as Section 2 requires. */
typedef struct {
    double alpha, beta, delta, mu;
} lll_nig;

typedef struct lll_ctx lll_ctx;

/* lll_init -- build a model context (Sections 2 and 4).
 *   out        : receives the context (set to NULL on failure).
 *   N          : accrual dates, N >= 2 (n = N-1 simulated rates), N <= 4096.
 *   tenor_delta: accrual fraction delta > 0 (all periods equal).
 *   L0         : [N] initial forward rates L(0, T_m), m = 0..N-1, all > 0
 *                (Eq. (i-val) gives them from the bond curve).
 *   steps_per_period: s >= 1.
 *   lambda     : [n*s][n], lambda[k*n + (l-1)] = lambda(t_k, T_l), the
 *                volatility of rate l at the left point of step k (LR1).
 *   driver     : lll_driver.
 *   nig        : NIG parameters (ignored for the Brownian driver); alpha > |beta|,
 *                delta > 0.
 *   Q, nodes, weights: quadrature of the Levy measure, Q in [1, 128]:
 *                int g(x) F(dx) ~= sum_j weights[j] g(nodes[j]) / nodes[j]^2,
 *                i.e. the weights integrate against x^2 nu(x) dx.  Nodes must be
 *                finite and non-zero.  Ignored (may be NULL, Q = 0) for the
 *                Brownian driver.
 *   cuda_stream: cudaStream_t to issue all work on (NULL = default stream).
 * Builds in FP64 on the GPU the per-step tables of the compensator integrand
 * and the frozen-curve drift b(t_k, T_l; Z(0)) of Eq. (Picard-2) with its
 * running integral.  Returns LLL_EDOMAIN (context usable) when
 * max_k sum_l |lambda(t_k, T_l)| >= alpha - |beta|. */
int lll_init(lll_ctx **out, int N, double tenor_delta, const double *L0, int steps_per_period,
             const double *lambda, int driver, lll_nig nig, int Q, const double *nodes,
             const double *weights, void *cuda_stream);

/* lll_set_product -- the payoff recorded at every T_m (m = 1..n) for the
 * strikes of lll_set_strikes; takes effect at the next simulation.
 *   LLL_PRODUCT_CAPLET (0, default): the caplet of Eq. (caplet) on L(T_m, T_m).
 *   LLL_PRODUCT_SWAPTION (1): the co-terminal payer swaption expiring at T_m
 *     on the swap over [T_m, T_N] (fixed rate K against L, both legs paying at
 *     T_{m+1} .. T_N), a multi-LIBOR derivative (Section 1): its value at T_m
 *     is (1 - B(T_m,T_N) - K delta sum_{j>m} B(T_m,T_j))^+, priced under the
 *     terminal measure as B(0,T_N) E[((1 + delta L_m) P - 1 - K delta S)^+]
 *     with P = prod_{l>m} (1 + delta L_l(T_m)) and S = sum_{j=m+1}^{N}
 *     prod_{l>=j} (1 + delta L_l(T_m)) (FP64 on the GPU).  lll_price_caplets
 *     then returns swaption prices.  The batched launch prices caplets only. */
#define LLL_PRODUCT_CAPLET 0
#define LLL_PRODUCT_SWAPTION 1
int lll_set_product(lll_ctx *ctx, int product);

/* lll_set_strikes -- strikes of the caplets of Eq. (caplet), needed before
 * lll_simulate because payoffs are accumulated on the fly.
 *   n_strikes: 1..64; strikes: [n][n_strikes], row m-1 = caplet fixing at T_m. */
int lll_set_strikes(lll_ctx *ctx, int n_strikes, const double *strikes);

/* lll_set_snapshots -- keep log L_l(T_m), l >= m, for `count` paths of each
 * simulation (parity checks): the paths whose index relative to first_path is
 * a multiple of `stride` (>= 1), the first `count` of them.  count = 0
 * disables. */
int lll_set_snapshots(lll_ctx *ctx, uint64_t count, uint64_t stride);

/* lll_simulate -- simulate paths [first_path, first_path + paths) of one
 * scheme and accumulate caplet payoff sums.  Path p draws its increments from
 * Philox-4x32-10 with key (seed_lo, seed_hi) and counter (k, 0, p_lo, p_hi),
 * so any path range reproduces the same paths (sharding, resumption).  Resets
 * the accumulators.  Asynchronous on the context's stream.
 * LLL_MLP requires lll_mlp_train or lll_mlp_load first (LLL_ESTATE). */
int lll_simulate(lll_ctx *ctx, int scheme, uint64_t first_path, uint64_t paths, uint64_t seed);

/* lll_get_sums -- FP64 payoff sums of the last simulation, for merging shards
 * in a fixed order: sum[n][n_strikes], sumsq[n][n_strikes], *count = paths.
 * Synchronises the stream. */
int lll_get_sums(lll_ctx *ctx, double *sum, double *sumsq, uint64_t *count);

/* lll_price_caplets -- Eq. (caplet): price = mean payoff (already carries
 * delta * B(0, T_N) and the numeraire product), stderr = sample standard
 * deviation / sqrt(paths).  prices, stderr_: [n][n_strikes].  stderr_ may be
 * NULL.  Synchronises the stream. */
int lll_price_caplets(lll_ctx *ctx, double *prices, double *stderr_);

/* lll_get_paths -- snapshots of the last simulation: out[(p*n + (m-1))*n +
 * (l-1)] = log L_l(T_m) for l >= m (NaN for l < m), for recorded snapshots
 * p in [first, first+count); recorded snapshot q is path first_path +
 * q*stride.  Synchronises the stream. */
int lll_get_paths(lll_ctx *ctx, uint64_t first, uint64_t count, float *out);

/* lll_set_launch -- override the launch shape of the path kernels:
 * threads per block (32..256, multiple of 32), resident blocks per SM
 * (0 = occupancy maximum), table rows staged per pipeline chunk (>= 1),
 * paths carried per thread (1 or 2, one-lane mapping only; 2 is compiled for
 * Q <= 64 and shares each staged table load between two paths), lanes per
 * path (1: one lane sweeps all nodes of its path; 2 or 4: a group of that
 * many lanes shares the node sweep of as many paths, full and Picard with the
 * NIG driver).  0 for any argument selects the library default. */
int lll_set_launch(lll_ctx *ctx, int threads_per_block, int blocks_per_sm, int chunk_rows,
                   int paths_per_thread, int lanes_per_path);

/* lll_set_mapping -- how the full and Picard schemes map a path onto lanes.
 *   LLL_MAP_PATH (0, default): one lane carries a path (or a lane group of
 *     lll_set_launch shares the node sweep of as many paths) and sweeps its
 *     live rates from the last one down, sharing the suffix products of the
 *     beta factors between rates.
 *   LLL_MAP_TENOR (1): tenor-parallel (Section 3.1-3.2: under the Picard
 *     iterate of Eq. (Picard-2) every (path, tenor) evolves on its own):
 *     `lanes` (4, 8, 16 or 32) lanes share a path, lane g owning the rate
 *     block n - g r .. n - (g+1) r + 1, r = ceil(n / lanes) rounded up to odd.
 *     Each lane multiplies the beta factors of its block per node, a
 *     multiplicative scan over the lanes gives every lane the product over
 *     the blocks above, and each lane sweeps and steps its own rates.  About
 *     5/3 of the one-lane arithmetic plus the scan, for `lanes` times the
 *     threads per path: for small path budgets.  128-thread blocks; caplet
 *     payoffs and a node table only (LLL_EUNSUPPORTED otherwise at simulation).
 *   LLL_MAP_STEP (2, Picard only; `lanes` ignored): the Euler steps of a path
 *     evaluated in parallel.  Under Eq. (Picard-2) the drift at t_k reads
 *     Z^(1)(t_k), a function of the driving path alone, so after a prefix
 *     sum of lambda_l Delta H over the steps, one thread per (step, path) runs
 *     the suffix sweep of that step, and a second prefix sum over the steps
 *     gives the log-rates at every maturity.  Same arithmetic per unit as the
 *     path mapping; intermediate arrays of about 4 (S + 2 S n + n^2) bytes per
 *     path, processed in chunks within 2 GiB of device memory.  For small
 *     path budgets (a single term structure of 2^12 paths).  LLL_FULL
 *     returns LLL_EUNSUPPORTED under it: the full scheme's drift reads the
 *     simulated rates, so its steps are sequential.  lll_simulate_noalloc
 *     ignores it (path mapping).
 * Other schemes ignore the mapping. */
#define LLL_MAP_PATH 0
#define LLL_MAP_TENOR 1
#define LLL_MAP_STEP 2
int lll_set_mapping(lll_ctx *ctx, int mapping, int lanes);

/* lll_kernel_ms -- device time of the last simulation's path kernel and of the
 * whole lll_simulate call, from CUDA events on the context's stream.
 * Synchronises the stream. */
int lll_kernel_ms(lll_ctx *ctx, float *path_kernel_ms, float *simulate_ms);

/* lll_simulate_noalloc -- lll_simulate for callers that must not allocate
 * device memory once they are running: services that reserve all their device
 * memory at start-up through their own pool, and latency-bound callers that
 * cannot afford the device-wide synchronisation cudaMalloc / cudaFree may
 * imply.  (The paper has no counterpart: this is an engineering entry point.)
 *   ctx, first_path, paths, seed: as for lll_simulate (snapshots are not
 *                recorded).
 *   scheme     : LLL_FULL, LLL_PICARD or LLL_FROZEN; LLL_MLP, LLL_EXPAND1 and
 *                LLL_EXPAND2 return LLL_EUNSUPPORTED (their kernels keep
 *                per-context buffers), any other value LLL_EINVAL.
 *   d_sums     : caller-owned device buffer of n * n_strikes * 2 doubles,
 *                d_sums[2*(m*n_strikes + q)] = sum of payoffs and [... + 1] =
 *                sum of squared payoffs of maturity m+1, strike q.
 * Makes the same launch as lll_simulate, so the sums equal lll_get_sums'.
 * Scratch (per-block path state and payoff partials) comes from one static
 * 32 MiB device array that every GPU loading the library holds until exit;
 * a launch needing more returns LLL_EUNSUPPORTED with the byte counts in
 * lll_last_error.  Each call made outside a stream capture looks the array's
 * address up (cudaGetSymbolAddress), so a module reloaded after
 * cudaDeviceReset is found at its new address; a call made while the
 * context's stream is captured uses the address the last uncaptured call
 * found on that device, so make one uncaptured call first (a captured first
 * call returns LLL_ESTATE).
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads, other contexts on the same device) race and corrupt each
 * other's results; serialise them.  Nothing in the array needs clearing
 * between calls.  Asynchronous on the context's stream. */
int lll_simulate_noalloc(lll_ctx *ctx, int scheme, uint64_t first_path, uint64_t paths,
                         uint64_t seed, double *d_sums);

/* lll_build_nig_quadrature -- Q-point Gauss rule of the weight x^2 nu(x) on
 * [-xmax, xmax], nu the NIG Levy density (Barndorff-Nielsen 1997; the paper
 * gives only kappa, Section 4).  Host computation in FP64.
 *   nodes, weights: [Q] outputs, Q in [1, 128]. */
int lll_build_nig_quadrature(lll_nig nig, double xmax, int Q, double *nodes, double *weights);

/* ---- Batches of independent term structures -------------------------------
 * Many models (uneven tenor counts, curves, volatilities, NIG parameters,
 * strike grids and path budgets) simulated by one persistent launch: the
 * resident blocks claim work items (runs of one instance's 128-path tiles) in
 * order of decreasing cost until none is left, and each instance's results
 * are summed in tile order, so they are the same from launch to launch
 * whatever block ran which item.  Instance q draws its increments
 * from Philox counter (k, q, p_lo, p_hi): independent streams per instance.
 * All instances must use the NIG driver and the same padded Q (16, 32, 64, 96
 * or 128). */
typedef struct {
    int N;                 /* accrual dates (as lll_init) */
    double tenor_delta;
    const double *L0;      /* [N] */
    int steps_per_period;
    const double *lambda;  /* [n*s][n] */
    int driver;            /* LLL_DRIVER_NIG */
    lll_nig nig;
    int Q;
    const double *nodes, *weights; /* [Q] */
    int n_strikes;
    const double *strikes; /* [n][n_strikes] */
    uint64_t paths;        /* > 0 */
} lll_instance;

typedef struct lll_batch lll_batch;

/* lll_batch_init -- build every instance (FP64 tables on the GPU, as lll_init;
 * an instance's LLL_EDOMAIN warning is accepted).  Inputs are copied. */
int lll_batch_init(lll_batch **out, int n_inst, const lll_instance *inst, void *cuda_stream);

/* lll_batch_set_launch -- the launch shape of scheme LLL_FULL or LLL_PICARD
 * (-1: both): threads per block (0: 128), blocks per SM (0: occupancy
 * maximum), table rows per staged chunk (0: default) and paths per thread
 * (0 or 1: one; 2: two paths share every staged table load, for padded
 * Q <= 64).  Each scheme keeps its own shape, schedule and graph: alternating
 * schemes rebuilds nothing; a new shape rebuilds that scheme's on its next
 * simulation.  Synchronises the stream.  LLL_EINVAL for values out of range;
 * an unsupported combination is reported by the next lll_batch_simulate
 * (LLL_EUNSUPPORTED). */
int lll_batch_set_launch(lll_batch *b, int scheme, int threads_per_block, int blocks_per_sm, int chunk_rows,
                         int paths_per_thread);

/* lll_batch_use_graph -- enable: the first simulation of a scheme captures
 * its launch sequence (descriptor upload from pinned memory, reset of the
 * work-item counter, batch kernel, final reduction) in a CUDA graph; later
 * ones replay it. */
int lll_batch_use_graph(lll_batch *b, int enable);

/* lll_batch_simulate -- all instances, scheme LLL_FULL or LLL_PICARD, one
 * launch.  Asynchronous. */
int lll_batch_simulate(lll_batch *b, int scheme, uint64_t seed);

/* lll_batch_prices -- caplet prices and standard errors of instance q
 * ([n_q][n_strikes_q]).  Synchronises the stream. */
int lll_batch_prices(lll_batch *b, int q, double *prices, double *stderr_);

/* lll_batch_set_snapshots -- parity snapshots of instance q, as
 * lll_set_snapshots does for one context: log L_l(T_m) (l >= m) of `count`
 * paths of that instance, those whose index is a multiple of `stride`,
 * recorded by every following lll_batch_simulate (count = 0 disables).
 * Allocates the instance's snapshot buffer; synchronises the stream. */
int lll_batch_set_snapshots(lll_batch *b, int q, uint64_t count, uint64_t stride);

/* lll_batch_get_paths -- snapshots of instance q from the last batch
 * simulation, laid out as lll_get_paths: out[(p*n_q + (m-1))*n_q + (l-1)],
 * recorded snapshot p = path p*stride of the instance.  Synchronises. */
int lll_batch_get_paths(lll_batch *b, int q, uint64_t first, uint64_t count, float *out);

/* lll_batch_kernel_ms -- device time of the last lll_batch_simulate. */
int lll_batch_kernel_ms(lll_batch *b, float *ms);

void lll_batch_destroy(lll_batch *b);

/* ---- Learned compensator (the MLP drift of LLL_MLP) -----------------------
 * A SiLU multilayer perceptron stands in for the jump integral of
 * Eq. (LIBOR-drift-PT) in the full scheme.  Input row (in_dim = N + 3):
 *   (t / T_N, i / n, lambda(t, T_i) * s_lam, u_0 .. u_{N-1}),
 *   u_m = (log L_m(t) - log L_m(0)) * s_u,
 * output f with A_i = C_i + s_y f, where C_i is the compensator with all later
 * weights zero (exact, from the FP64 tables).  BF16 weights and activations,
 * FP32 accumulation (tensor cores), FP32 master weights, Adam.  Parameters
 * are one flat FP32 vector: for each hidden layer W (hidden x in) and b,
 * then the output w (outputs x hidden) and b (outputs); lll_mlp_layout gives
 * the offsets.
 * Vector head (head = 1): one evaluation per (path, Euler step) gives every
 * rate's compensator: input (t s_t, u_0 .. u_{N-1}), outputs = n padded to 16
 * (column i - 1 for rate i; rates already fixed are ignored), trained on the
 * same records with the MSE over their live rates.  LLL_MLP then runs a
 * tcgen05 vector-head kernel -- hidden 128 with n <= 48, or hidden 256 with
 * n <= 121, input width <= 128 and at most 16 strikes (the whole simulation
 * in one persistent launch, the weights streamed from L2) -- or, for other
 * networks, layer by layer (LLL_MLP_KERNEL_LAYERED), at about 1/n of the
 * per-rate cost. */
typedef struct {
    int hidden;           /* width of every hidden layer: 128 or 256 */
    int layers;           /* hidden layers: 1..4 */
    uint64_t train_paths; /* full-scheme (quadrature) paths simulated to make the data */
    int records_per_path; /* Euler steps recorded per path (1..8), one pair per live rate each */
    int epochs;           /* passes over the pairs (head 1: over the records) */
    int batch;            /* rows per Adam step (>= 32) */
    double lr, lr_final;  /* Adam step size, decayed geometrically to lr_final (<= 0: constant) */
    uint64_t seed;
    int head;             /* 0: one output per (step, rate); 1: vector head */
} lll_mlp_cfg;

/* lll_mlp_init -- a fresh network (He-uniform weights from `seed`, zero
 * biases) with the context's feature scales; s_y = 1 until trained. */
int lll_mlp_init(lll_ctx *ctx, int hidden, int layers, uint64_t seed);
/* The same with the output head chosen (0 per rate, 1 vector). */
int lll_mlp_init_head(lll_ctx *ctx, int hidden, int layers, int head, uint64_t seed);
/* lll_mlp_shape -- head (0/1) and output width of the context's network. */
int lll_mlp_shape(lll_ctx *ctx, int *head, int *outputs);

/* lll_mlp_train -- generate training pairs with the quadrature full scheme on
 * the GPU (paths keyed by cfg->seed, not by pricing seeds), set s_y to the RMS
 * target, and train with Adam on the GPU.  *final_loss = MSE of the last batch
 * in units of s_y^2.  Synchronises the stream. */
int lll_mlp_train(lll_ctx *ctx, const lll_mlp_cfg *cfg, double *final_loss);

/* lll_mlp_layout -- parameter count, input width, padded input width and the
 * flat offsets (W_0, b_0, ..., W_{L-1}, b_{L-1}, w_out, b_out: 2L+2 values). */
int lll_mlp_layout(lll_ctx *ctx, size_t *n_params, int *in_dim, int *in_pad, size_t *offsets);

/* lll_mlp_params -- direction 0: copy the FP32 parameters and the five scales
 * (s_t, s_i, s_lam, s_u, s_y) out; 1: copy them in (either pointer may be
 * NULL).  count must equal the parameter count. */
int lll_mlp_params(lll_ctx *ctx, int direction, float *params, size_t count, float *scales);

/* lll_mlp_eval -- run the network on host feature rows x[rows][in_dim]:
 * out[rows * outputs] (may be NULL).  With targets y[rows]: *loss = mean (f - y)^2, and
 * with grads != NULL its gradient w.r.t. every parameter (flat layout). */
int lll_mlp_eval(lll_ctx *ctx, const float *x, const float *y, int rows, float *out, float *grads,
                 double *loss);

/* lll_mlp_set_kernel -- which kernel runs LLL_MLP:
 *   LLL_MLP_KERNEL_AUTO (0, default): the tensor-memory kernel where it
 *     supports the network, else the warp-level one;
 *   LLL_MLP_KERNEL_WARP (1): warp-level mma.sync (hidden 128, N <= 61);
 *   LLL_MLP_KERNEL_TC (2): tcgen05 with TMEM accumulators, hidden 128 and
 *     2..4 layers, where its shared-memory plan (weights, feature rows and
 *     the CTA's path state) fits: N <= 61 with 3 layers, N <= 66 with 2, and
 *     N <= 54 with 4 layers and 5 strikes (fewer with more strikes); the
 *     vector head needs n <= 48 with hidden 128, or hidden 256, 2..4 layers,
 *     n <= 121 and at most 16 strikes.  Its waits are bounded, and a wait
 *     that gives up makes the next read of the results return LLL_ETIMEOUT;
 *   LLL_MLP_KERNEL_LAYERED (3): any network (hidden 256, N up to 125): per
 *     Euler step, the rows (path, live rate) of a chunk of up to 2^20 rows go
 *     through the network layer by layer with the training GEMMs; AUTO takes
 *     it when neither fused kernel fits.
 * A fused choice the network does not fit returns LLL_EUNSUPPORTED at
 * simulation. */
#define LLL_MLP_KERNEL_AUTO 0
#define LLL_MLP_KERNEL_WARP 1
#define LLL_MLP_KERNEL_TC 2
#define LLL_MLP_KERNEL_LAYERED 3
int lll_mlp_set_kernel(lll_ctx *ctx, int kind);

/* lll_set_gemm_kernel -- the tensor-core kernel of the learned compensator's
 * GEMMs (training: forward, dX and split-K dW; LLL_MLP_KERNEL_LAYERED
 * inference), for the whole process:
 *   LLL_GEMM_TC (0, default): tcgen05.mma, operands in shared memory
 *     (128-byte swizzle), FP32 accumulator in tensor memory, 128 x N tiles
 *     (N = 64, 128 or 256), bounded waits (a wait that gives up makes
 *     lll_mlp_train return LLL_ETIMEOUT);
 *   LLL_GEMM_MMA_SYNC (1): the warp-level mma.sync.m16n8k16 kernel.
 * Both compute the same products with FP32 accumulation (in different
 * orders).  Not thread-safe against concurrent training in other threads. */
#define LLL_GEMM_TC 0
#define LLL_GEMM_MMA_SYNC 1
int lll_set_gemm_kernel(int kind);

/* lll_gemm_bf16 -- one product of the kernel lll_set_gemm_kernel selected,
 * on host buffers (for tests of the GEMM itself; allocates and frees device
 * memory and synchronises the device).  BF16 operands as raw bits:
 *   C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = A[m*lda+k] (ta = 0) or
 *   A[k*lda+m] (ta = 1), B(k,n) = B[k*ldb+n] (tb = 0) or B[n*ldb+k] (tb = 1).
 *   epi 0: C = the product (split-K over `splits` ranges, added in order);
 *   epi 1 (ta = 0, tb = 1, the forward layer): C = z = product + bias[n],
 *          H = bf16(SiLU(z)), SiLU(z) = z (1 + tanh(z/2)) / 2;
 *   epi 2 (ta = 0, tb = 0, the backward layer): C = d = product *
 *          SiLU'(Zin[m][n]), H = bf16(d);
 *   epi 3 / 4 (ta = 0, tb = 1, tcgen05 only): C = product + bias[n] /
 *          product + bias[m] (the vector head's output layer, computed
 *          transposed in the layered inference).
 * C, Zin: [M][N] FP32; H: [M][N] BF16 bits; bias: [N] ([M] for epi 4).  The paper has no
 * counterpart: the GEMMs serve the learned compensator. */
int lll_gemm_bf16(int ta, int tb, int epi, const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N,
                  int K, int splits, const float *bias, const float *Zin, float *C, uint16_t *H);

/* lll_inject -- failure-detection testing: LLL_INJECT_MMA_STALL makes the
 * next launch of the tensor-memory MLP kernel issue no MMAs, so that its
 * bounded waits run out (about 2 s): the launch ends by itself, frees its
 * tensor memory, and the next lll_get_sums / lll_price_caplets returns
 * LLL_ETIMEOUT; the context stays usable.  No GPU fault is involved.
 * LLL_INJECT_NONE clears a pending injection. */
#define LLL_INJECT_NONE 0
#define LLL_INJECT_MMA_STALL 1
int lll_inject(lll_ctx *ctx, int what);

/* ---- Measuring calls -------------------------------------------------------
 * lll_philox_words -- the device Philox-4x32-10 of every path kernel (Salmon
 * et al., SC'11; the generator behind the driver increments of Section 4)
 * evaluated on caller counters, for bit-exact checks of the integer stream:
 *   ctr  : [count][4] host counters (word 0 .. word 3; the path kernels use
 *          (step, instance, path_lo, path_hi)),
 *   seed : key (seed_lo, seed_hi),
 *   out  : [count][4] host output words.
 * count in [1, 2^24].  Allocates and frees device memory on the current
 * device and synchronises it. */
int lll_philox_words(const uint32_t *ctr, uint64_t count, uint64_t seed, uint32_t *out);

/* lll_measure_pipe_rates -- results per SM per clock of the instructions the
 * rooflines are stated in, measured on the current device (one block of 32
 * warps per SM, 8 independent chains per thread, SM cycle counter; median
 * over the SMs).  rates[0] tanh.approx.f32, [1] ex2.approx.ftz.f32,
 * [2] rcp.approx.ftz.f32, [3] FP32 lane-ops of packed fma.rn.f32x2 (two per
 * lane), [4] FP32 lane-ops of scalar fma.rn.f32; the first `count` (1..5)
 * are measured.  Takes a few milliseconds; synchronises the device.  The
 * paper has no counterpart: the numbers are the denominators of the
 * benchmark's roofline fractions. */
int lll_measure_pipe_rates(double *rates, int count);

/* lll_mlp_save / lll_mlp_load -- flat binary file: magic, (hidden, layers,
 * in_dim, N), the five scales, parameter count, FP32 parameters. */
int lll_mlp_save(lll_ctx *ctx, const char *path);
int lll_mlp_load(lll_ctx *ctx, const char *path);

/* lll_last_error -- message of the last failing call on ctx (ctx may be NULL:
 * the last failure of lll_init or lll_build_nig_quadrature in this thread). */
const char *lll_last_error(const lll_ctx *ctx);

/* lll_destroy -- free the context and its device memory (NULL is a no-op). */
void lll_destroy(lll_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LLL_H */
