// Integer throughput of the device, measured: the denominator of the integer
// (ALU) roofline of the path sweep.  The paper's aggregation (Eq. 1) is a
// chain of additions and minima on small unsigned losses; this kernel runs
// 16 independent chains of one such instruction per thread, on every SM,
// and counts scalar operations (a packed two-lane 16-bit instruction counts
// as two).
#include "rsgm_internal.cuh"

namespace rsgm {
namespace {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;

__device__ unsigned g_peak_sink[1024];  // written only if a chain hits the seed: keeps the chains live

template <int KIND>
__device__ __forceinline__ void op(unsigned &x, unsigned y)
{
    if (KIND == RSGM_PEAK_I32_ADD) asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(y));
    if (KIND == RSGM_PEAK_I32_MIN) asm volatile("min.u32 %0, %0, %1;" : "+r"(x) : "r"(y));
    if (KIND == RSGM_PEAK_U16X2_MIN) asm volatile("min.u16x2 %0, %0, %1;" : "+r"(x) : "r"(y));
    if (KIND == RSGM_PEAK_U16X2_MIX) {
        // the mix of Eq. 1 on packed pairs: a minimum, then an addition
        asm volatile("min.u16x2 %0, %0, %1;" : "+r"(x) : "r"(y));
        asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(y));
    }
}

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, unsigned seed)
{
    unsigned r[kChains];
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kChains; ++j) r[j] = (t * 2654435761u) ^ (seed + 977u * j);
    for (int i = 0; i < iters; ++i) {
        const unsigned y = (unsigned)i | 0x00010001u;
#pragma unroll
        for (int j = 0; j < kChains; ++j) op<KIND>(r[j], y);
    }
    unsigned acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc ^= r[j];
    if (acc == seed) g_peak_sink[t & 1023] = acc;
}

template <int KIND>
cudaError_t run_peak(int blocks, int iters, cudaStream_t st)
{
    k_peak<KIND><<<blocks, kPeakThreads, 0, st>>>(iters, 0x9E3779B9u);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_peak(int kind, int blocks, int iters, cudaStream_t st)
{
    switch (kind) {
    case RSGM_PEAK_I32_ADD: return run_peak<RSGM_PEAK_I32_ADD>(blocks, iters, st);
    case RSGM_PEAK_I32_MIN: return run_peak<RSGM_PEAK_I32_MIN>(blocks, iters, st);
    case RSGM_PEAK_U16X2_MIN: return run_peak<RSGM_PEAK_U16X2_MIN>(blocks, iters, st);
    case RSGM_PEAK_U16X2_MIX: return run_peak<RSGM_PEAK_U16X2_MIX>(blocks, iters, st);
    default: return cudaErrorInvalidValue;
    }
}

// Scalar integer operations one launch performs.
double peak_ops(int kind, int blocks, int iters)
{
    const double instr = (double)blocks * kPeakThreads * (double)iters * kChains;
    switch (kind) {
    case RSGM_PEAK_I32_ADD:
    case RSGM_PEAK_I32_MIN: return instr;
    case RSGM_PEAK_U16X2_MIN: return 2.0 * instr;
    case RSGM_PEAK_U16X2_MIX: return 2.0 * 2.0 * instr;  // two packed instructions per step
    default: return 0.0;
    }
}

int peak_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_peak<RSGM_PEAK_I32_ADD>, kPeakThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 2048 / kPeakThreads;
    }
    return n > 0 ? n : 1;
}

}  // namespace rsgm
