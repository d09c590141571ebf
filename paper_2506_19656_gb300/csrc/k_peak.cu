// k_peak.cu -- device microbenchmarks of the instruction sequences that the
// roofline fractions are quoted against (measurement only, not a step of the
// method).
//
// Each thread runs kChains accumulation chains for `iters` rounds.  An
// operation's first operand is the accumulator of the next chain, a value
// carried around the loop, so no compiler stage can hoist a loop-invariant
// part out of the loop (ptxas did, for a subtraction of two invariant
// floats) or fold a chain of identical additions into a multiplication; the
// operations are inline PTX marked volatile.  The values themselves are
// meaningless (the floats may overflow; the timing does not depend on it).
// A full grid (every SM at its thread limit) keeps enough warps in flight
// for issue, not latency, to bound the rate.
//   kind 0: abs-diff-accumulate as one integer sad.s32 (the ALU pipe)
//   kind 1: abs-diff-accumulate on the FP32 pipe: sub.f32, then add.f32 of
//           its absolute value (exact for 10-bit samples stored as floats)
//   kind 2: the mix of two kind-0 and one kind-1 abs-diff per three
//   kind 3: 32-bit integer multiply-add (mad.lo.s32), the transform's unit
#include <cuda_runtime.h>

#include <cstdint>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kChains = 12;  // a multiple of 3 (kind 2 takes chains in threes)
constexpr int kPeakThreads = 256;

__device__ __forceinline__ void sad_op(uint32_t& acc, uint32_t a, uint32_t b) {
    asm volatile("sad.s32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(b));
}
__device__ __forceinline__ void fad_op(float& acc, float a, float b) {
    asm volatile("{\n\t.reg .f32 t;\n\tsub.f32 t, %1, %2;\n\tabs.f32 t, t;\n\tadd.f32 %0, %0, t;\n\t}"
                 : "+f"(acc) : "f"(a), "f"(b));
}
__device__ __forceinline__ void mad_op(uint32_t& acc, uint32_t a, uint32_t b) {
    asm volatile("mad.lo.s32 %0, %1, %2, %0;" : "+r"(acc) : "r"(a), "r"(b));
}

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(const uint32_t* __restrict__ in, int iters,
                                                        uint32_t* __restrict__ sink) {
    const int t = threadIdx.x & 63;
    uint32_t a[kChains], b[kChains], acc[kChains];
    float fb[kChains], facc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        a[k] = in[(t + k) & 63];
        b[k] = in[64 + ((t + 3 * k) & 63)];
        acc[k] = a[k];
        fb[k] = __uint_as_float(b[k]);
        facc[k] = __uint_as_float(a[k]);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const int n = (k + 1) % kChains;  // the next chain's accumulator is the first operand
            if (KIND == 0) sad_op(acc[k], acc[n], b[k]);
            if (KIND == 1) fad_op(facc[k], facc[n], fb[k]);
            if (KIND == 2) {  // the next chain of the same kind: chains 3j + 2 are FP32, the rest integer
                if (k % 3 == 2) fad_op(facc[k], facc[(k + 3) % kChains], fb[k]);
                else sad_op(acc[k], acc[(k + 1) % 3 == 2 ? (k + 2) % kChains : n], b[k]);
            }
            if (KIND == 3) mad_op(acc[k], acc[n], b[k]);
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k] + __float_as_uint(facc[k]);
    if (s == 0x9e3779b9u) sink[blockIdx.x] = s;  // keeps the chains live; practically never stored
}

}  // namespace

int peak_chains() { return kChains; }

cudaError_t launch_peak(int kind, const uint32_t* in, int iters, uint32_t* sink, int* threads_out,
                        cudaStream_t st) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void (*fn)(const uint32_t*, int, uint32_t*) = kind == 0 ? k_peak<0> : kind == 1 ? k_peak<1> : kind == 2 ? k_peak<2>
                                                                                                           : k_peak<3>;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kPeakThreads, 0);
    if (e != cudaSuccess) return e;
    if (per < 1) per = 1;
    const int grid = sms * per;
    *threads_out = grid * kPeakThreads;
    fn<<<grid, kPeakThreads, 0, st>>>(in, iters, sink);
    return cudaGetLastError();
}

}  // namespace xvh
