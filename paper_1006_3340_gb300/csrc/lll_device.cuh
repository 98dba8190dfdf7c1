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

// Discounted payoff (under the terminal measure, times B(0, T_N)) at T_m for
// strike K.  Caplet, Eq. (caplet): delta B(0,T_N) prod_{l>m} (1 + delta L_l) (L_m - K)^+.
// Co-terminal payer swaption on the swap over [T_m, T_N]: its value at T_m is
// (1 - B(T_m,T_N) - K delta sum_{j>m} B(T_m,T_j))^+, and divided by the
// numeraire B(T_m, T_N) it is ((1 + delta L_m) P - 1 - K delta S)^+.
__device__ __forceinline__ double payoff(const PathArgs &a, double P, double S, float Lm, float K)
{
    if (a.product == 0) return (double)(a.dBN * (float)P * fmaxf(Lm - K, 0.0f));
    const double X = (1.0 + (double)(a.delta * Lm)) * P - 1.0 - (double)K * (double)a.delta * S;
    return X > 0.0 ? (double)a.dBN / (double)a.delta * X : 0.0;
}

}  // namespace lll
