// lll_device.cuh -- device-side random numbers and driver increments.
//
// Philox-4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3" (SC'11).  The NIG increment (Section 4 of the paper draws
// its NIG driver by the usual normal variance-mean mixture, without detail)
// is beta V + sqrt(V) Z + mu h with V ~ IG(mean m, shape l),
// m = dbar h / gamma, l = (dbar h)^2; V by Michael, Schucany & Haas (1976).
#pragma once

#include <cstdint>

#include "lll_internal.h"

namespace lll {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Top 23 bits of a word as an odd multiple of 2^-24 in (0, 1); exact in FP32.
__device__ __forceinline__ float u01(uint32_t w)
{
    return fmaf((float)(w >> 9), 1.0f / 8388608.0f, 1.0f / 16777216.0f);
}

__device__ __forceinline__ double u01d(uint32_t w)
{
    return fma((double)(w >> 9), 1.0 / 8388608.0, 1.0 / 16777216.0);
}

// Driver increment of path p over step k.  Counter (k, inst, p_lo, p_hi),
// key (seed_lo, seed_hi).  Box-Muller z1 = r cos(2 pi u1), z2 = r sin(2 pi u1),
// r = sqrt(-2 log u0); z1^2 feeds the IG draw, z2 is the mixing normal.
//
// The IG acceptance test u2 <= m / (m + y) picks one of two roots; a flip
// changes the increment completely, so near its threshold the decision is
// re-taken in FP64 from the same uniforms (the precision of the reference
// computation).  Away from the threshold FP32 cannot flip it: the FP32 error
// of the threshold is below 1e-6 relative and the re-check band is 4e-5.
__device__ __forceinline__ float draw_increment(const PathArgs &a, uint64_t p, uint32_t k)
{
    const uint4 w = philox4x32_10(make_uint4(k, a.inst, (uint32_t)p, (uint32_t)(p >> 32)), a.key0,
                                  a.key1);
    const float u0 = u01(w.x), u1 = u01(w.y);
    const float r = sqrtf(-2.0f * logf(u0));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    const float z1 = r * cs;
    if (a.driver == 1) return a.sqrt_h * z1;
    const float z2 = r * sn;
    const float nu = z1 * z1;
    const float mnu = a.ig_m * nu;
    const float ypl = fmaf(a.ig_hl, mnu + sqrtf(fmaf(a.ig_fl, nu, mnu * mnu)), a.ig_m);
    const float y = a.ig_m2 / ypl;
    const float thr = a.ig_m / (a.ig_m + y);
    const float u2 = u01(w.z);
    bool take_small = u2 <= thr;
    if (fabsf(u2 - thr) < 4e-5f * thr + 1e-7f) {
        const double u0d = u01d(w.x), u1d = u01d(w.y), u2d = u01d(w.z);
        const double rd = sqrt(-2.0 * log(u0d));
        const double z1d = rd * cospi(2.0 * u1d);
        const double nud = z1d * z1d;
        const double md = a.ig_md, ld = a.ig_ld;
        const double yp = md + md * md * nud / (2.0 * ld) +
                          md / (2.0 * ld) * sqrt(4.0 * md * ld * nud + md * md * nud * nud);
        const double yd = md * md / yp;
        take_small = u2d <= md / (md + yd);
    }
    const float V = take_small ? y : ypl;
    return fmaf(a.nig_beta, V, fmaf(sqrtf(V), z2, a.nig_muh));
}

// Payoff quantities of one path at T_m from its log-rates z(i) = log L_i(T_m),
// i = m..n (z is a callable): L_m, P = prod_{l>m} (1 + delta L_l) and, for
// swaptions, S = 1 + sum_{j=m+1}^{n} prod_{l>=j} (1 + delta L_l), i.e.
// B(T_m, T_j) / B(T_m, T_N) summed over the payment dates T_{m+1} .. T_N.
// Caplets keep P in FP32 (a product of factors near 1, multiplied by a
// non-negative payoff); swaptions keep P and S in FP64 (each factor formed as
// 1 + fl32(delta L)), because their payoff subtracts 1 from them.
template <class ZF>
__device__ __forceinline__ void maturity_products(const PathArgs &a, int m, ZF z, double &P, double &S, float &Lm)
{
    if (a.product == 0) {
        float Pf = 1.0f;
        for (int i = a.n; i > m; --i) Pf *= fmaf(a.delta, expf(z(i)), 1.0f);
        P = (double)Pf;
        S = 1.0;
    } else {
        P = 1.0;
        S = 1.0;
        for (int i = a.n; i > m; --i) {
            P *= 1.0 + (double)(a.delta * expf(z(i)));
            S += P;
        }
    }
    Lm = expf(z(m));
}

// The same quantities, with the factors (1 + delta L_i) of eight rates at a
// time computed ahead of their place in the sequential product: the same
// operations in the same order (a factor past m is 1, an exact product), so
// the results are identical, while the loads and exponentials of a group
// overlap instead of forming one dependent chain.
template <class ZF>
__device__ __forceinline__ void maturity_products_grouped(const PathArgs &a, int m, ZF z, double &P, double &S,
                                                          float &Lm)
{
    if (a.product == 0) {
        float Pf = 1.0f;
        for (int i0 = a.n; i0 > m; i0 -= 8) {
            float f[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) f[u] = i0 - u > m ? fmaf(a.delta, expf(z(i0 - u)), 1.0f) : 1.0f;
#pragma unroll
            for (int u = 0; u < 8; ++u) Pf *= f[u];
        }
        P = (double)Pf;
        S = 1.0;
    } else {
        P = 1.0;
        S = 1.0;
        for (int i0 = a.n; i0 > m; i0 -= 8) {
            double f[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) f[u] = i0 - u > m ? 1.0 + (double)(a.delta * expf(z(i0 - u))) : 1.0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 - u > m) {
                    P *= f[u];
                    S += P;
                }
        }
    }
    Lm = expf(z(m));
}

// Caplet payoff, Eq. (caplet), discounted under the terminal measure:
// delta B(0,T_N) prod_{l>m} (1 + delta L_l) (L_m - K)^+, with P the product.
// An FP32 number.
__device__ __forceinline__ float caplet_payoff(const PathArgs &a, float P, float Lm, float K)
{
    return a.dBN * P * fmaxf(Lm - K, 0.0f);
}

// Discounted payoff (under the terminal measure, times B(0, T_N)) at T_m for
// strike K.  Caplet: caplet_payoff.
// Co-terminal payer swaption on the swap over [T_m, T_N]: its value at T_m is
// (1 - B(T_m,T_N) - K delta sum_{j>m} B(T_m,T_j))^+, and divided by the
// numeraire B(T_m, T_N) it is ((1 + delta L_m) P - 1 - K delta S)^+.
__device__ __forceinline__ double payoff(const PathArgs &a, double P, double S, float Lm, float K)
{
    if (a.product == 0) return (double)caplet_payoff(a, (float)P, Lm, K);
    const double X = (1.0 + (double)(a.delta * Lm)) * P - 1.0 - (double)K * (double)a.delta * S;
    return X > 0.0 ? (double)a.dBN / (double)a.delta * X : 0.0;
}

// ---- A warp's payoff sums without FP64 arithmetic --------------------------
// GB300 issues FP64 arithmetic at about 1/64 of the FP32 rate (1.25 against
// 80 TFLOP/s nominal), and a warp's sums of its paths' payoffs and squared
// payoffs, formed at every maturity for every strike, are the path kernels'
// only FP64 work per path (ncu: the FP64 pipe 8 % busy in the Picard path
// kernel on the N = 40 workload when they were FP64 sums).  Caplet payoffs are FP32
// numbers, so their sums are kept as unevaluated pairs hi + lo of FP32
// numbers ("double-float"):
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2) gives the exact rounding error of an
//    FP32 addition;
//  * the FMA form of Dekker's product (Dekker 1971) gives v * v exactly as
//    fl(v v) + fma(v, v, -fl(v v));
//  * after each addition the pair is renormalised by Dekker's Fast2Sum.
// Adding two pairs this way has a relative error below 3 * 2^-48 when both
// have one sign (Joldes, Muller and Popescu 2017, "Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic"); payoffs are
// non-negative, so the five levels of the butterfly keep a warp's sums within
// about 6e-14 of the exact ones.  The block reduction adds the warps' pairs
// the same way and turns the result into FP64 (hi + lo) once per strike and
// maturity.
struct DFloat {
    float hi, lo;
};

__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ DFloat df_square(float v)
{
    const float p = v * v;
    return {p, fmaf(v, v, -p)};
}

__device__ __forceinline__ DFloat df_warp_sum(DFloat v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, DFloat{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
}

// Sums over the warp of the caplet payoffs v of every lane's paths (0 for a
// path that is not simulated) and of v^2: (sum hi, sum lo, sum2 hi, sum2 lo),
// the same on every lane.
__device__ __forceinline__ float4 caplet_warp_sums_inline(DFloat s1, DFloat s2)
{
    s1 = df_warp_sum(s1);
    s2 = df_warp_sum(s2);
    return make_float4(s1.hi, s1.lo, s2.hi, s2.lo);
}

// The same as calls.  They stay out of line on purpose: inlined into the
// path kernel, this code (like a plain FP32 shuffle sum in its place) changed
// the code generated for the kernel's rate sweep, which then ran 7 % slower
// (Picard, N = 40 workload, 2^20 paths: 64.3 ms inlined, 59.7 ms as a call,
// 60.3 ms with the former FP64 sums).
static __device__ __noinline__ float4 caplet_warp_sums1(float v)
{
    return caplet_warp_sums_inline(DFloat{v, 0.0f}, df_square(v));
}

static __device__ __noinline__ float4 caplet_warp_sums2(float v0, float v1)
{
    return caplet_warp_sums_inline(df_add(DFloat{v0, 0.0f}, DFloat{v1, 0.0f}), df_add(df_square(v0), df_square(v1)));
}

template <int R>
__device__ __forceinline__ float4 caplet_warp_sums(const float (&v)[R])
{
    static_assert(R == 1 || R == 2, "one or two paths per lane");
    if constexpr (R == 1) return caplet_warp_sums1(v[0]);
    else return caplet_warp_sums2(v[0], v[1]);
}

// The sums over warps 0 .. nw-1 of a block for strike q, from the block's
// reduction buffer of 16-byte slots [warp][ns] (caplets: the four floats of
// caplet_warp_sums, added as pairs in warp order and turned into FP64 once;
// swaptions: the FP64 sums of v and v^2, added in warp order).
__device__ __forceinline__ void block_payoff_sums(const PathArgs &a, const double *red, int nw, int ns, int q,
                                                  double &s1, double &s2)
{
    if (a.product == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(red);
        float4 r = r4[q];
        DFloat x{r.x, r.y}, y{r.z, r.w};
        for (int wv = 1; wv < nw; ++wv) {
            r = r4[(size_t)wv * ns + q];
            x = df_add(x, DFloat{r.x, r.y});
            y = df_add(y, DFloat{r.z, r.w});
        }
        s1 = (double)x.hi + (double)x.lo;
        s2 = (double)y.hi + (double)y.lo;
    } else {
        s1 = 0.0;
        s2 = 0.0;
        for (int wv = 0; wv < nw; ++wv) {
            s1 += red[2 * ((size_t)wv * ns + q) + 0];
            s2 += red[2 * ((size_t)wv * ns + q) + 1];
        }
    }
}

}  // namespace lll
