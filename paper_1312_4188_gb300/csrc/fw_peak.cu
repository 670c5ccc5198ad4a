// Integer throughput microbenchmark: the measured denominator of the INT32
// roofline that the rule-check rates are reported against.
//
// Every thread runs eight interleaved chains of 32-bit integer instructions
// with no memory traffic inside the timed loop (one store per thread at the
// end keeps the chains live). Each chain step reads the chain's own value and
// its neighbour's, so no step can be folded into another, and sixteen warps
// per scheduler hide each instruction's latency. Three instruction mixes:
//   kind 0  lop3 only (3-input logic, the integer ALU pipe),
//   kind 1  mad.lo.u32 only (integer multiply-add, which the FMA pipe issues),
//   kind 2  the two alternated 1:1 (both pipes fed: the issue limit).
// The rule-check kernels mix both kinds (logic tests and compares on the ALU
// pipe, the port offsets as multiply-adds), so kind 2 is the roof they are
// measured against and kind 0 tells how far the ALU pipe alone goes.
#include <climits>

#include "fw_internal.cuh"

namespace fwk {

constexpr int kPeakChains = 8;
constexpr int kPeakRounds = 16;  // chain steps per loop trip: kPeakChains * kPeakRounds = 128 ops

__device__ __forceinline__ uint32_t peak_lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ uint32_t peak_mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(512) k_int32_peak(uint32_t *__restrict__ sink, int iters, uint32_t seed) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = seed * (2u * j + 1u) ^ (tid * 0x9E3779B9u + j);
    const uint32_t m = (seed | 1u) ^ (tid << 1);  // runtime multiplier (odd)
    for (int i = 0; i < iters; ++i) {
        const uint32_t x = (uint32_t)i ^ seed;
#pragma unroll
        for (int r = 0; r < kPeakRounds; ++r) {
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) {
                const uint32_t nb = a[(j + 1) % kPeakChains];
                if (KIND == 0 || (KIND == 2 && (j & 1) == 0)) a[j] = peak_lop3(a[j], nb, x);
                else a[j] = peak_mad(a[j], m, nb);
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) acc ^= a[j];
    sink[tid] = acc;
}

}  // namespace fwk

using namespace fwk;

extern "C" int fw_int32_peak_launch(int kind, int32_t iters, int32_t blocks, int32_t threads, uint32_t *sink,
                                    void *stream, int64_t *ops_per_launch) {
    if (kind < 0 || kind > 2 || iters < 1 || iters > (1 << 24) || blocks < 1 || blocks > (1 << 20) ||
        threads < 32 || threads > 512 || threads % 32 != 0 || sink == nullptr || ops_per_launch == nullptr)
        return set_status(FW_EINVAL);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t seed = 0x2545F491u;
    if (kind == 0) k_int32_peak<0><<<blocks, threads, 0, st>>>(sink, iters, seed);
    else if (kind == 1) k_int32_peak<1><<<blocks, threads, 0, st>>>(sink, iters, seed);
    else k_int32_peak<2><<<blocks, threads, 0, st>>>(sink, iters, seed);
    *ops_per_launch = (int64_t)blocks * threads * iters * (kPeakChains * kPeakRounds);
    return set_status(cuda_status(cudaGetLastError()));
}
