// lll_tc.cuh -- device helpers of the tcgen05 kernels: shared-memory operand
// descriptors (K-major, 128-byte swizzle), mbarriers with bounded waits,
// tensor-memory loads, TMA tile loads and the products.
//
// Operand layout: a 64-wide K block of an R-row BF16 operand is R rows of
// 128 bytes; the 16-byte chunk c8 of row r sits at
//   (r / 8) 1024 + (r mod 8) 128 + ((c8 xor (r mod 8)) 16),
// the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B and a box of 64
// elements, and the one the descriptor sdesc() describes.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lll {
namespace tc {

constexpr long long kWaitBudget = 4000000000ll; // clock cycles (about 2 s) before a wait gives up

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t a)
{
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_m128(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Byte offset of the 16-byte chunk c8 (0..7) of row r within a 64-wide K block.
__device__ __forceinline__ uint32_t swz(int r, int c8)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c8 ^ (r & 7)) << 4));
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint32_t mbar_test(uint32_t a, uint32_t par)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(a), "r"(par)
                 : "memory");
    return ok;
}

__device__ __forceinline__ uint32_t mbar_try(uint32_t a, uint32_t par)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(a), "r"(par)
                 : "memory");
    return ok;
}

// One thread waits for the completion of the phase of parity `par`.  Gives
// up when the CTA's abort word is set or after kWaitBudget cycles (then sets
// it and the launch's error word).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t par, volatile int *abort, int *err)
{
    const uint32_t a = saddr(b);
    if (mbar_test(a, par)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(a, par)) return true;
        if (*abort) return false;
        if (clock64() - t0 > kWaitBudget) {
            *abort = 1;
            atomicOr(err, 1);
            return false;
        }
    }
}

// The same for a whole warp, with warp-uniform decisions, so that the warp
// stays converged for the .sync.aligned tcgen05 instructions that follow.
__device__ __forceinline__ bool warp_wait(uint64_t *b, uint32_t par, volatile int *abort, int *err)
{
    const uint32_t a = saddr(b);
    if (__all_sync(0xffffffffu, mbar_test(a, par))) return true;
    const long long t0 = clock64();
    while (true) {
        if (__all_sync(0xffffffffu, mbar_try(a, par))) return true;
        const bool stop = *abort || clock64() - t0 > kWaitBudget;
        if (__any_sync(0xffffffffu, stop)) {
            if ((threadIdx.x & 31) == 0 && !*abort) {
                *abort = 1;
                atomicOr(err, 1);
            }
            return false;
        }
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols));
}

// D (tensor memory) = A B (+ D when acc != 0), both operands in shared memory.
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

// The same with A in tensor memory: at addresses 128 lanes (rows) x 8 columns,
// each column two BF16 values of consecutive K (lower K in the low half).
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t at, uint64_t bd, uint32_t id, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                 "r"(at), "l"(bd), "r"(id), "r"(acc));
}

// 8 columns of this thread's TMEM lane from r[0..7]; complete at tmem_wait_st.
__device__ __forceinline__ void tmem_st8(uint32_t ta, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Arrive on b once every product issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
                 : "memory");
}

// 2D TMA tile load of box {x .. x + bx - 1, y .. y + by - 1} into dst,
// completion counted in bytes on bar.  x * 2 bytes must be a multiple of 16;
// y may lie outside the tensor (those rows are filled with zeros).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const void *tmap)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// Accumulator columns of this thread's TMEM lane: the loads are issued by
// tmem_ld16 / tmem_ld8 and their registers become valid at tmem_wait, which
// takes them as in/out operands so that no use is scheduled before it.
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(ta));
}

__device__ __forceinline__ void tmem_ld8(uint32_t ta, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(ta));
}

#define LLL_TC_R16(r) "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), \
    "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])

#define LLL_TC_R8(r) "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])

__device__ __forceinline__ void tmem_wait8(uint32_t *r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : LLL_TC_R8(r) : : "memory");
}

__device__ __forceinline__ void tmem_wait(uint32_t *r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : LLL_TC_R16(r) : : "memory");
}

__device__ __forceinline__ void tmem_wait32(uint32_t *r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : LLL_TC_R16(r), LLL_TC_R16((r + 16)) : : "memory");
}

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
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

}  // namespace tc
}  // namespace lll
