// ludax_peak.cu -- integer-issue microbenchmark behind the playout roofline.
//
// The fused playouts are bitboard code: 3-input logic ops (LOP3), adds
// (IADD3) and funnel shifts (SHF) on 32-bit halves of the boards, plus the
// multiplies of the random draws.  Their roofline takes the SM's issue rate
// (4 warp instructions per clock per SM) and, for the pipe that executes
// these ops, half of it.  This kernel measures what a stream of one such op
// (or of two ops on alternate chains) reaches on this GPU: every thread
// keeps 8 independent chains (so latency is hidden by ILP as well as by
// the full occupancy of the grid), each step one inline-PTX instruction
// that the compiler cannot merge or drop.
#include <cuda_runtime.h>

#include "ludax_internal.cuh"

namespace {

constexpr int PEAK_THREADS = 256, PEAK_BLOCKS_PER_SM = 8, PEAK_CHAINS = 8;

// KIND 0 LOP3, 1 IADD, 2 SHF, 3 IMAD (multiply-add), 4 IMAD.HI (high half
// of the product), 5 LOP3 and IMAD on alternate chains (whether the two
// pipes issue side by side)
template <int KIND>
__device__ __forceinline__ void op(uint32_t& a, uint32_t b, uint32_t c, int chain) {
    if constexpr (KIND == 0) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a) : "r"(b), "r"(c));
    else if constexpr (KIND == 1) asm volatile("add.u32 %0, %0, %1;" : "+r"(a) : "r"(b));
    else if constexpr (KIND == 2) asm volatile("shf.l.wrap.b32 %0, %0, %1, %2;" : "+r"(a) : "r"(b), "r"(c));
    else if constexpr (KIND == 3) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a) : "r"(b), "r"(c));
    else if constexpr (KIND == 4) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a) : "r"(b));
    else if (chain & 1) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a) : "r"(b), "r"(c));
    else asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a) : "r"(b), "r"(c));
}

template <int KIND>
__global__ void __launch_bounds__(PEAK_THREADS) int_peak_kernel(long long iters, uint32_t* sink) {
    uint32_t a[PEAK_CHAINS];
    const uint32_t b = threadIdx.x * 0x9E3779B9u + 1u, c = blockIdx.x | 3u;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = b ^ (uint32_t)i;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < PEAK_CHAINS; ++i) op<KIND>(a[i], b, c, i);
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) x ^= a[i];
    if (x == 0x12345678u) sink[blockIdx.x] = x;  // keeps the chains live; practically never taken
}

__device__ uint32_t g_peak_sink[1];

}  // namespace

extern "C" {

int ludax_int_peak(int32_t kind, int64_t iters, int64_t* ops_out, void* stream) {
    if (kind < 0 || kind > 5 || iters < 1 || iters > (1ll << 30)) return LUDAX_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    uint32_t* sink = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), g_peak_sink) != cudaSuccess) return LUDAX_ERR_CUDA;
    const int grid = sms * PEAK_BLOCKS_PER_SM;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
        case 0: int_peak_kernel<0><<<grid, PEAK_THREADS, 0, s>>>(iters, sink); break;
        case 1: int_peak_kernel<1><<<grid, PEAK_THREADS, 0, s>>>(iters, sink); break;
        case 2: int_peak_kernel<2><<<grid, PEAK_THREADS, 0, s>>>(iters, sink); break;
        case 3: int_peak_kernel<3><<<grid, PEAK_THREADS, 0, s>>>(iters, sink); break;
        case 4: int_peak_kernel<4><<<grid, PEAK_THREADS, 0, s>>>(iters, sink); break;
        default: int_peak_kernel<5><<<grid, PEAK_THREADS, 0, s>>>(iters, sink); break;
    }
    if (ops_out) *ops_out = (int64_t)grid * PEAK_THREADS * PEAK_CHAINS * iters;
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

}  // extern "C"
