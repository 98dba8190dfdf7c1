// lll_mlp_path.cu -- the full scheme with the learned compensator (LLL_MLP).
//
// Same Euler scheme as the quadrature path kernel (Eq. (log-LIB-SDE-2) with
// the drift of Eq. (LIBOR-drift-PT)), but the jump compensator of every live
// rate comes from the trained network: A_i = C_i + s_y f(x_i), with the
// feature row x_i = (t s_t, i s_i, lambda_i s_lam, u_0 .. u_{N-1}) built from
// the simulated log-rates at t_k.
//
// Layout: one warp carries 32 paths (one per lane, state in the block's global
// scratch slot as in the quadrature kernel) and evaluates the network for them
// as two 16-row tiles on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulators).  The accumulator fragment of one layer is exactly the
// operand fragment of the next, so activations never leave registers; only
// the t / i / lambda columns of the first layer change from rate to rate and
// are patched into k-tile 0.  Weights are staged once per block in shared
// memory in fragment order (one 64-bit load per lane per mma).  The network's
// output for (path, rate) reaches the lane that owns the path through a small
// per-warp buffer; that lane then makes the Euler step and the caplet
// bookkeeping exactly like the quadrature kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lll_device.cuh"
#include "lll_internal.h"
#include "lll_mlp.h"

namespace lll {
namespace {

constexpr int kH = 128;          // hidden width handled by this kernel
constexpr int kNT = kH / 8;      // n-tiles per layer
constexpr int kKT = kH / 16;     // k-tiles of a hidden layer
constexpr int kWarps = 8;        // warps per block (256 paths per tile)

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16(x)); }

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float silu_t(float z) { return 0.5f * z * (1.0f + tanh_approx(0.5f * z)); }

__device__ __forceinline__ void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                    uint2 b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

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

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

struct MlpSmem {
    uint2 *wf;      // fragment-ordered B operands, all layers
    float *bias;    // [L][H]
    float *wout;    // [H] (BF16 values)
    __nv_bfloat16 *U; // [warps][32][upitch]
    float *D;       // [warps][n][32] network outputs
    double *bsum;   // [n * ns][4]
    double *red;    // [warps][ns][2]
};

__host__ __device__ inline size_t wf_count(int L, int KT0) { return (size_t)(KT0 + (L - 1) * kKT) * kNT * 32; }

__host__ __device__ inline size_t mlp_smem_bytes(int L, int KT0, int n, int ns)
{
    const int upitch = KT0 * 16 + 8;
    size_t b = al16(sizeof(uint2) * wf_count(L, KT0));
    b += al16(sizeof(float) * L * kH);
    b += al16(sizeof(float) * kH);
    b += al16(sizeof(__nv_bfloat16) * kWarps * 32 * upitch);
    b += al16(sizeof(float) * kWarps * n * 32);
    b += al16(sizeof(double) * 4 * n * ns);
    b += al16(sizeof(double) * 2 * kWarps * ns);
    return b;
}

template <int L, int KT0>
__global__ void __launch_bounds__(kWarps * 32, 1) mlp_path_kernel(const PathArgs a, const MlpArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = kWarps * 32;
    const int gq = lane >> 2, tq = lane & 3;
    const int n = a.n, s = a.s, S = a.S, ns = a.ns;
    constexpr int upitch = KT0 * 16 + 8;
    MlpSmem sm;
    {
        size_t o = 0;
        sm.wf = reinterpret_cast<uint2 *>(smem_raw + o); o += al16(sizeof(uint2) * wf_count(L, KT0));
        sm.bias = reinterpret_cast<float *>(smem_raw + o); o += al16(sizeof(float) * L * kH);
        sm.wout = reinterpret_cast<float *>(smem_raw + o); o += al16(sizeof(float) * kH);
        sm.U = reinterpret_cast<__nv_bfloat16 *>(smem_raw + o); o += al16(sizeof(__nv_bfloat16) * kWarps * 32 * upitch);
        sm.D = reinterpret_cast<float *>(smem_raw + o); o += al16(sizeof(float) * kWarps * n * 32);
        sm.bsum = reinterpret_cast<double *>(smem_raw + o); o += al16(sizeof(double) * 4 * n * ns);
        sm.red = reinterpret_cast<double *>(smem_raw + o);
    }
    // Stage the weights in fragment order: B(k, n) = W_l[n][k].
    const int in_pad = KT0 * 16;
    for (size_t e = tid; e < wf_count(L, KT0); e += T) {
        const int ln = (int)(e % 32);
        size_t rest = e / 32;
        const int nt = (int)(rest % kNT);
        rest /= kNT;
        int kt = (int)rest, l = 0, din = in_pad;
        if (kt >= KT0) { kt -= KT0; l = 1 + kt / kKT; kt %= kKT; din = kH; }
        const __nv_bfloat16 *W = g.wh + g.offW[l];
        const int col = nt * 8 + (ln >> 2), k0 = kt * 16 + (ln & 3) * 2;
        const __nv_bfloat16 *wr = W + (size_t)col * din;
        __nv_bfloat162 lo, hi;
        lo.x = wr[k0]; lo.y = wr[k0 + 1]; hi.x = wr[k0 + 8]; hi.y = wr[k0 + 9];
        sm.wf[e] = make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
    }
    for (int e = tid; e < L * kH; e += T) sm.bias[e] = g.wp[g.offb[e / kH] + e % kH];
    for (int e = tid; e < kH; e += T) sm.wout[e] = __bfloat162float(g.wh[g.off_wout + e]);
    for (int e = tid; e < 4 * n * ns; e += T) sm.bsum[e] = 0.0;
    __nv_bfloat16 *Uw = sm.U + (size_t)warp * 32 * upitch;
    float *Dw = sm.D + (size_t)warp * n * 32;
    for (int e = lane; e < 32 * upitch; e += 32) Uw[e] = __float2bfloat16(0.0f);
    const float b_out = g.wp[g.off_bout];
    const uint2 *wf0 = sm.wf;
    __syncthreads();

    float *st = a.state + (size_t)blockIdx.x * n * T + tid;
    const uint64_t ntiles = (a.paths + T - 1) / T;
    const float h = a.h;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t lp = tile * (uint64_t)T + tid;
        const bool active = lp < a.paths;
        const uint64_t p = a.first_path + lp;
        uint64_t sidx = ~0ull;
        if (a.snap != nullptr && active && lp % a.snap_stride == 0 && lp / a.snap_stride < a.n_snap)
            sidx = lp / a.snap_stride;
        for (int l = 0; l < n; ++l) st[(size_t)l * T] = 0.0f;

        for (int k = 0; k < S; ++k) {
            const int imin = k / s + 1;
            const bool mat = (k + 1) % s == 0;
            const float dH = draw_increment(a, p, (uint32_t)k);
            // features of this lane's path: u_m, m = 1..n at columns 4..3+n (u_0 = 0)
            __syncwarp();
            for (int m = 1; m <= n; ++m) Uw[lane * upitch + 3 + m] = __float2bfloat16(st[(size_t)(m - 1) * T] * g.sc.u_scale);
            __syncwarp();
            const float xt = (float)k * h * g.sc.t_scale;
#pragma unroll 1
            for (int mt = 0; mt < 2; ++mt) {
                uint32_t ua[KT0][4];
#pragma unroll
                for (int kt = 0; kt < KT0; ++kt) {
                    const __nv_bfloat16 *r0 = Uw + (size_t)(mt * 16 + gq) * upitch + kt * 16 + tq * 2;
                    const __nv_bfloat16 *r1 = r0 + 8 * upitch;
                    ua[kt][0] = *reinterpret_cast<const uint32_t *>(r0);
                    ua[kt][1] = *reinterpret_cast<const uint32_t *>(r1);
                    ua[kt][2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
                    ua[kt][3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
                }
#pragma unroll 1
                for (int i = imin; i <= n; ++i) {
                    const float lam = a.row[(size_t)k * n + (i - 1)].x;
                    if (tq == 0) ua[0][0] = ua[0][1] = pack2(xt, (float)i * g.sc.i_scale);
                    else if (tq == 1) ua[0][0] = ua[0][1] = pack2(lam * g.sc.lam_scale, 0.0f);
                    float acc[kNT][4];
                    uint32_t af[kKT][4];
                    // layer 0
#pragma unroll
                    for (int nt = 0; nt < kNT; ++nt) {
                        const float b0 = sm.bias[nt * 8 + tq * 2], b1 = sm.bias[nt * 8 + tq * 2 + 1];
                        acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
                    }
#pragma unroll
                    for (int kt = 0; kt < KT0; ++kt)
#pragma unroll
                        for (int nt = 0; nt < kNT; ++nt)
                            mma(acc[nt], ua[kt][0], ua[kt][1], ua[kt][2], ua[kt][3], wf0[(kt * kNT + nt) * 32 + lane]);
                    // hidden layers 1 .. L-1
#pragma unroll
                    for (int l = 1; l < L; ++l) {
#pragma unroll
                        for (int kt = 0; kt < kKT; ++kt) {
                            af[kt][0] = pack2(silu_t(acc[2 * kt][0]), silu_t(acc[2 * kt][1]));
                            af[kt][1] = pack2(silu_t(acc[2 * kt][2]), silu_t(acc[2 * kt][3]));
                            af[kt][2] = pack2(silu_t(acc[2 * kt + 1][0]), silu_t(acc[2 * kt + 1][1]));
                            af[kt][3] = pack2(silu_t(acc[2 * kt + 1][2]), silu_t(acc[2 * kt + 1][3]));
                        }
                        const uint2 *wl = sm.wf + (size_t)(KT0 + (l - 1) * kKT) * kNT * 32;
#pragma unroll
                        for (int nt = 0; nt < kNT; ++nt) {
                            const float b0 = sm.bias[l * kH + nt * 8 + tq * 2];
                            const float b1 = sm.bias[l * kH + nt * 8 + tq * 2 + 1];
                            acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
                        }
#pragma unroll
                        for (int kt = 0; kt < kKT; ++kt)
#pragma unroll
                            for (int nt = 0; nt < kNT; ++nt)
                                mma(acc[nt], af[kt][0], af[kt][1], af[kt][2], af[kt][3], wl[(kt * kNT + nt) * 32 + lane]);
                    }
                    // output layer on BF16 activations
                    float o0 = 0.0f, o1 = 0.0f;
#pragma unroll
                    for (int nt = 0; nt < kNT; ++nt) {
                        const float w0 = sm.wout[nt * 8 + tq * 2], w1 = sm.wout[nt * 8 + tq * 2 + 1];
                        o0 = fmaf(bf16r(silu_t(acc[nt][0])), w0, o0);
                        o0 = fmaf(bf16r(silu_t(acc[nt][1])), w1, o0);
                        o1 = fmaf(bf16r(silu_t(acc[nt][2])), w0, o1);
                        o1 = fmaf(bf16r(silu_t(acc[nt][3])), w1, o1);
                    }
                    o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
                    o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
                    o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
                    o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
                    if (tq == 0) {
                        Dw[(size_t)(i - 1) * 32 + mt * 16 + gq] = o0 + b_out;
                        Dw[(size_t)(i - 1) * 32 + mt * 16 + gq + 8] = o1 + b_out;
                    }
                }
            }
            __syncwarp();
            // Euler step of this lane's path with A_i = C_i + s_y f
            for (int i = n; i >= imin; --i) {
                const size_t row = (size_t)k * n + (i - 1);
                const float lam = a.row[row].x;
                const float A = g.Ctab[row] + g.sc.y_scale * Dw[(size_t)(i - 1) * 32 + lane];
                float *sp = st + (size_t)(i - 1) * T;
                const float z = sp[0] + fmaf(lam, dH, -A * h);
                sp[0] = z;
                if (mat && sidx != ~0ull)
                    a.snap[((size_t)(imin - 1) * n + (i - 1)) * a.snap_pitch + sidx] = z + a.Z0[i - 1];
            }
            if (mat) {
                const int m = imin;
                double Pp, Sp;
                float Lm;
                maturity_products(a, m, [&](int i) { return st[(size_t)(i - 1) * T] + a.Z0[i - 1]; }, Pp, Sp, Lm);
                for (int q = 0; q < ns; ++q) {
                    const float K = a.strikes[(size_t)(m - 1) * ns + q];
                    const double pay = active ? payoff(a, Pp, Sp, Lm, K) : 0.0;
                    const double s1 = warp_sum(pay);
                    const double s2 = warp_sum(pay * pay);
                    if (lane == 0) {
                        sm.red[((size_t)warp * ns + q) * 2 + 0] = s1;
                        sm.red[((size_t)warp * ns + q) * 2 + 1] = s2;
                    }
                }
                __syncthreads();
                if (tid < ns) {
                    double s1 = 0.0, s2 = 0.0;
                    for (int wv = 0; wv < kWarps; ++wv) {
                        s1 += sm.red[((size_t)wv * ns + tid) * 2 + 0];
                        s2 += sm.red[((size_t)wv * ns + tid) * 2 + 1];
                    }
                    double *acc = sm.bsum + 4 * ((size_t)(m - 1) * ns + tid);
                    kahan_add(acc + 0, acc + 1, s1);
                    kahan_add(acc + 2, acc + 3, s2);
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * n * ns * 2;
    for (int e = tid; e < n * ns; e += T) {
        out[2 * e + 0] = sm.bsum[4 * e + 0];
        out[2 * e + 1] = sm.bsum[4 * e + 2];
    }
}

typedef void (*MlpKernelFn)(const PathArgs, const MlpArgs);

template <int L>
MlpKernelFn pick_kt(int KT0)
{
    switch (KT0) {
    case 1: return mlp_path_kernel<L, 1>;
    case 2: return mlp_path_kernel<L, 2>;
    case 3: return mlp_path_kernel<L, 3>;
    case 4: return mlp_path_kernel<L, 4>;
    default: return nullptr;
    }
}

MlpKernelFn pick_mlp(int L, int KT0)
{
    switch (L) {
    case 1: return pick_kt<1>(KT0);
    case 2: return pick_kt<2>(KT0);
    case 3: return pick_kt<3>(KT0);
    case 4: return pick_kt<4>(KT0);
    default: return nullptr;
    }
}

}  // namespace

int mlp_path_threads() { return kWarps * 32; }

size_t mlp_path_smem(int layers, int in_pad, int n, int ns) { return mlp_smem_bytes(layers, in_pad / 16, n, ns); }

bool mlp_path_supported(int hidden, int layers, int in_pad)
{
    return hidden == kH && pick_mlp(layers, in_pad / 16) != nullptr && in_pad % 16 == 0;
}

int mlp_path_occupancy(int layers, int in_pad, size_t smem, int *blocks_per_sm)
{
    MlpKernelFn f = pick_mlp(layers, in_pad / 16);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kWarps * 32, smem);
}

int launch_mlp_path(int layers, int in_pad, int grid, size_t smem, cudaStream_t st, const PathArgs &a,
                    const MlpArgs &g)
{
    MlpKernelFn f = pick_mlp(layers, in_pad / 16);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, kWarps * 32, smem, st>>>(a, g);
    return (int)cudaGetLastError();
}

}  // namespace lll
