// lll_probe.cu -- two measuring entry points: the device Philox words, and the
// per-SM issue rates of the instructions the rooflines are stated in.
//
// lll_philox_words evaluates the Philox-4x32-10 of the path kernels
// (lll_device.cuh) on caller counters, so tests can compare every output word
// of the GPU generator with the oracle's and with an external generator.
//
// lll_measure_pipe_rates runs one block per SM (the shared-memory request
// keeps a second block off the SM) of 32 warps, each thread carrying 8
// independent dependency chains of one instruction, and times the block with
// the SM's cycle counter.  Results per SM per clock:
//   [0] tanh.approx.f32 (one per SiLU of the learned compensator),
//   [1] ex2.approx.ftz.f32, [2] rcp.approx.ftz.f32 (the weight w of a rate;
//       each followed by an FP32 add, which keeps the chain from folding),
//   [3] FP32 lane-ops of packed fma.rn.f32x2 (two per lane and instruction:
//       the sweep of the quadrature compensator issues these),
//   [4] FP32 lane-ops of scalar fma.rn.f32.
// The median over the SMs is returned.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lll.h"
#include "lll_device.cuh"
#include "lll_internal.h"

namespace lll {
namespace {

__global__ void philox_words_kernel(const uint4 *ctr, uint64_t count, uint32_t k0, uint32_t k1, uint4 *out)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = philox4x32_10(ctr[i], k0, k1);
}

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kProbeThreads = 1024;
constexpr size_t kProbeSmem = 160 * 1024; // one block per SM

enum Op { TANH = 0, EX2 = 1, RCP = 2, FFMA2 = 3, FFMA = 4 };

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) pipe_kernel(float seed, unsigned long long *cycles, float *sink)
{
    extern __shared__ float keep_sm_alone[];
    float v[kChains];
    float2 v2[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        v[c] = seed * (float)(threadIdx.x + c);
        v2[c] = make_float2(v[c], -v[c]);
    }
    const float2 a2 = make_float2(0.999f, 0.998f), b2 = make_float2(1e-3f, 2e-3f);
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == TANH) asm volatile("tanh.approx.f32 %0, %0;" : "+f"(v[c]));
            if (OP == EX2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
            // rcp(rcp(x)) could be folded by the assembler: an add between keeps
            // the chain (it issues to the FMA pipe, not the MUFU).
            if (OP == RCP) asm volatile("rcp.approx.ftz.f32 %0, %0;\n\tadd.f32 %0, %0, 0f3F800000;" : "+f"(v[c]));
            if (OP == FFMA) asm volatile("fma.rn.f32 %0, %0, 0f3F7FBE77, 0f3A83126F;" : "+f"(v[c]));
            if (OP == FFMA2) v2[c] = __ffma2_rn(v2[c], a2, b2);
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += (OP == FFMA2) ? v2[c].x + v2[c].y : v[c];
    if (acc == 12345.678f) sink[threadIdx.x] = acc + keep_sm_alone[0]; // never true; keeps the chains
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

typedef void (*PipeFn)(float, unsigned long long *, float *);

}  // namespace
}  // namespace lll

using namespace lll;

extern "C" int lll_philox_words(const uint32_t *ctr, uint64_t count, uint64_t seed, uint32_t *out)
{
    if (!ctr || !out || count == 0 || count > (1ull << 24))
        return record_error(nullptr, LLL_EINVAL, "need counters, outputs and 1 <= count <= 2^24");
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    const size_t bytes = sizeof(uint4) * count;
    cudaError_t e = cudaMalloc((void **)&d_ctr, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_out, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_ctr, ctr, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int T = 256;
        philox_words_kernel<<<(unsigned)((count + T - 1) / T), T>>>(d_ctr, count, (uint32_t)seed,
                                                                     (uint32_t)(seed >> 32), d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d_ctr);
    cudaFree(d_out);
    if (e != cudaSuccess) return record_error(nullptr, LLL_ECUDA, cudaGetErrorString(e));
    return LLL_OK;
}

extern "C" int lll_measure_pipe_rates(double *rates, int count)
{
    const PipeFn fns[] = {pipe_kernel<TANH>, pipe_kernel<EX2>, pipe_kernel<RCP>, pipe_kernel<FFMA2>,
                          pipe_kernel<FFMA>};
    const double per_instr[] = {1.0, 1.0, 1.0, 2.0, 1.0}; // lane-ops per lane and instruction
    const int nfn = (int)(sizeof(fns) / sizeof(fns[0]));
    if (!rates || count < 1 || count > nfn) return record_error(nullptr, LLL_EINVAL, "rates is NULL or count not in [1, 5]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long *d_cyc = nullptr;
    float *d_sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_cyc, sizeof(unsigned long long) * sms);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_sink, sizeof(float) * kProbeThreads);
    std::vector<unsigned long long> cyc(sms);
    for (int f = 0; f < count && e == cudaSuccess; ++f) {
        e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) { // the first launch warms up
            fns[f]<<<sms, kProbeThreads, kProbeSmem>>>(0.37f, d_cyc, d_sink);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e == cudaSuccess) e = cudaMemcpy(cyc.data(), d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        std::sort(cyc.begin(), cyc.end());
        const double ops = (double)kProbeThreads * kChains * kIters * per_instr[f];
        rates[f] = ops / (double)std::max<unsigned long long>(cyc[sms / 2], 1);
    }
    cudaFree(d_cyc);
    cudaFree(d_sink);
    if (e != cudaSuccess) return record_error(nullptr, LLL_ECUDA, cudaGetErrorString(e));
    return LLL_OK;
}
