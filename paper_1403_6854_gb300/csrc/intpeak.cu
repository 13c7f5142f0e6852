// Integer-pipe peak of this GPU, measured (the measurement helper behind the
// integer roofline of the scan kernels; the paper has no counterpart).
//
// The sorted sweep and the split walk are bound by integer issue, not by
// memory: their inner loops are logic ops (LOP3), byte permutes (PRMT),
// minima (IMNMX and the 16x2 SIMD VIMNMX), shifts, adds and population
// counts.  Each kernel below runs one of those operations in 8 independent
// dependency chains per thread (so that issue, not latency, limits it), as
// inline PTX so the operation is explicit, over a grid of resident CTAs on
// every SM, and reports operations per second (CUDA events around the
// launch) and operations per SM per cycle (clock64 inside each CTA).
#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/selscan_peak.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

template <int OP>
__device__ __forceinline__ unsigned op(unsigned a, unsigned b, unsigned c)
{
    unsigned r;
    switch (OP) {
    case SELSCAN_PEAK_LOP3:
        asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
        break;
    case SELSCAN_PEAK_PRMT:
        asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
        break;
    case SELSCAN_PEAK_IMNMX:
        asm volatile("min.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b ^ c));
        break;
    case SELSCAN_PEAK_VIMNMX2:
        asm volatile("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b ^ c));
        break;
    case SELSCAN_PEAK_POPC:
        asm volatile("popc.b32 %0, %1;" : "=r"(r) : "r"(a ^ b));
        r += c;
        break;
    case SELSCAN_PEAK_SHF:
        asm volatile("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
        break;
    default:   // SELSCAN_PEAK_IADD3
        asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        r += c;
        break;
    }
    return r;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) peak_kernel(int iters, unsigned seed, unsigned *sink,
                                                        long long *cycles)
{
    unsigned x[kChains];
    const unsigned t = threadIdx.x + blockIdx.x * blockDim.x;
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed * (t + 1u) + 0x9E3779B9u * (unsigned)(c + 1);
    const unsigned b = seed ^ t, cc = seed + 0x7F4A7C15u;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = op<OP>(x[c], b + (unsigned)c, cc);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    unsigned acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c];
    if (acc == 0x12345678u) sink[t] = acc;          // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
cudaError_t run(int ctas, int iters, unsigned *sink, long long *cycles, cudaStream_t s)
{
    peak_kernel<OP><<<ctas, kThreads, 0, s>>>(iters, 12345u, sink, cycles);
    return cudaGetLastError();
}

cudaError_t dispatch(int which, int ctas, int iters, unsigned *sink, long long *cycles,
                     cudaStream_t s)
{
    switch (which) {
    case SELSCAN_PEAK_LOP3: return run<SELSCAN_PEAK_LOP3>(ctas, iters, sink, cycles, s);
    case SELSCAN_PEAK_PRMT: return run<SELSCAN_PEAK_PRMT>(ctas, iters, sink, cycles, s);
    case SELSCAN_PEAK_IMNMX: return run<SELSCAN_PEAK_IMNMX>(ctas, iters, sink, cycles, s);
    case SELSCAN_PEAK_VIMNMX2: return run<SELSCAN_PEAK_VIMNMX2>(ctas, iters, sink, cycles, s);
    case SELSCAN_PEAK_POPC: return run<SELSCAN_PEAK_POPC>(ctas, iters, sink, cycles, s);
    case SELSCAN_PEAK_SHF: return run<SELSCAN_PEAK_SHF>(ctas, iters, sink, cycles, s);
    default: return run<SELSCAN_PEAK_IADD3>(ctas, iters, sink, cycles, s);
    }
}

// Operations counted per chain step: one, except for POPC and IADD3, whose
// chains also carry one add (counted too: the add keeps the chain dependent).
int ops_per_step_of(int which)
{
    return (which == SELSCAN_PEAK_POPC || which == SELSCAN_PEAK_IADD3) ? 2 : 1;
}

}  // namespace

extern "C" int selscan_peak_int(int32_t which, int32_t iters, void *scratch, size_t scratch_bytes,
                                selscan_peak_result *res)
{
    if (which < 0 || which >= SELSCAN_PEAK_NUM || iters < 1 || !scratch || !res)
        return SELSCAN_PEAK_ERR_ARG;
    int dev = 0, sms = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev) != cudaSuccess)
        return SELSCAN_PEAK_ERR_CUDA;
    // four 512-thread CTAs per SM: 64 warps, the most an SM holds
    const int ctas = 4 * sms;
    const size_t need = (size_t)ctas * kThreads * 4 + (size_t)ctas * 8;
    if (scratch_bytes < need || ((uintptr_t)scratch & 15)) return SELSCAN_PEAK_ERR_ARG;
    unsigned *sink = (unsigned *)scratch;
    long long *cycles = (long long *)((unsigned char *)scratch + (size_t)ctas * kThreads * 4);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return SELSCAN_PEAK_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return SELSCAN_PEAK_ERR_CUDA; }
    int rc = SELSCAN_PEAK_OK;
    float ms = 0.f;
    // one warm-up launch, then the timed one
    if (dispatch(which, ctas, iters, sink, cycles, 0) != cudaSuccess ||
        cudaEventRecord(a, 0) != cudaSuccess ||
        dispatch(which, ctas, iters, sink, cycles, 0) != cudaSuccess ||
        cudaEventRecord(b, 0) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
        rc = SELSCAN_PEAK_ERR_CUDA;
    long long host_cycles[4096];
    long long maxc = 0;
    if (rc == SELSCAN_PEAK_OK) {
        const int nc = ctas < 4096 ? ctas : 4096;
        if (cudaMemcpy(host_cycles, cycles, (size_t)nc * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SELSCAN_PEAK_ERR_CUDA;
        for (int i = 0; i < nc && rc == SELSCAN_PEAK_OK; ++i)
            if (host_cycles[i] > maxc) maxc = host_cycles[i];
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != SELSCAN_PEAK_OK) return rc;
    const double ops = (double)ctas * kThreads * (double)iters * 16.0 * kChains * ops_per_step_of(which);
    res->ops = ops;
    res->ms = ms;
    res->ops_per_s = ops / (ms * 1e-3);
    res->sms = sms;
    res->cycles = (double)maxc;
    // all CTAs are resident at once (four per SM), so each SM ran a quarter of the grid
    res->ops_per_sm_per_cycle = maxc > 0 ? ops / sms / (double)maxc : 0.0;
    res->clock_mhz_attr = clk_khz / 1000.0;
    res->clock_mhz_implied = maxc > 0 ? (double)maxc / (ms * 1e3) : 0.0;
    return SELSCAN_PEAK_OK;
}

extern "C" size_t selscan_peak_scratch_bytes(void)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    const int ctas = 4 * sms;
    return (size_t)ctas * kThreads * 4 + (size_t)ctas * 8;
}
