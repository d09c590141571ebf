// k_dec.cu -- the decoder's kernels: one frame of CUs for G groups per launch
// (the plain path; the batched path decodes in the persistent kernel), and
// the reconstruction back in the cube's units.
#include <cuda_runtime.h>

#include <cstdint>

#include "dec.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kNT = 256;
template <int N> constexpr int kMinBlocks = N == 64 ? 1 : (N == 32 ? 2 : 4);

template <int N>
__global__ void __launch_bounds__(kNT, kMinBlocks<N>)
k_dec_frame(const int16_t* __restrict__ levels, const uint16_t* __restrict__ ref, const int16_t* __restrict__ mv,
            const uint8_t* __restrict__ tu_log2, int64_t gstride, int Hp, int Wp, int qp, int64_t pu_gstride,
            uint16_t* recon, uint64_t* bits, int64_t bits_gstride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int cu = blockIdx.x, g = blockIdx.y, nx = Wp / N;
    const int64_t o = g * pu_gstride + cu;
    int mvx = 0, mvy = 0;
    if (ref) { mvx = mv[2 * o]; mvy = mv[2 * o + 1]; }
    const uint32_t b = xvd::dec_cu<N, kNT>(levels + g * gstride, ref ? ref + g * gstride : nullptr, (int64_t)Hp * Wp,
                                           Hp, Wp, (cu % nx) * N, (cu / nx) * N, mvx, mvy, tu_log2[o], qp,
                                           recon + g * gstride, smem);
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(bits + g * bits_gstride),
                                    (unsigned long long)b);
}

template <int N>
cudaError_t dec_n(const int16_t* levels, const uint16_t* ref, const int16_t* mv, const uint8_t* tu_log2, int G,
                  int64_t gstride, int Hp, int Wp, int qp, int64_t pu_gstride, uint16_t* recon, uint64_t* bits,
                  int64_t bits_gstride, cudaStream_t st) {
    const size_t smem = xvd::dec_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_dec_frame<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((Hp / N) * (Wp / N), G);
    k_dec_frame<N><<<grid, kNT, smem, st>>>(levels, ref, mv, tu_log2, gstride, Hp, Wp, qp, pu_gstride, recon, bits,
                                            bits_gstride);
    return cudaGetLastError();
}

// Band b (group b/3, channel b%3) over the valid H x W region: x^ = min + q
// (max - min)/1023 in double (multiply, then add), rounded to float32 -- from
// a per-band table of the 1024 values.  One warp per row; blockIdx.y = band.
constexpr int kUnpackThreads = 256;
__global__ void __launch_bounds__(kUnpackThreads)
k_unpack(const uint16_t* __restrict__ recon, int T, int H, int W, int Hp, int Wp, const double* __restrict__ mm,
         float* __restrict__ dst) {
    const int b = blockIdx.y, g = b / 3, c = b % 3;
    __shared__ float s_v[1024];
    const double lo = mm[2 * b], hi = mm[2 * b + 1];
    const double delta = __ddiv_rn(__dsub_rn(hi, lo), 1023.0);
    for (int v = threadIdx.x; v < 1024; v += kUnpackThreads)
        s_v[v] = __double2float_rn(__dadd_rn(lo, __dmul_rn((double)v, delta)));
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t rows = (int64_t)T * H;
    const int warps = (int)gridDim.x * (kUnpackThreads / 32);
    for (int64_t row = (int64_t)blockIdx.x * (kUnpackThreads / 32) + (threadIdx.x >> 5); row < rows; row += warps) {
        const int t = (int)(row / H), y = (int)(row - (int64_t)t * H);
        const uint16_t* src = recon + ((((int64_t)g * T + t) * 3 + c) * Hp + y) * Wp;
        float* out = dst + (((int64_t)b * T + t) * H + y) * W;
        for (int x = lane; x < W; x += 32) out[x] = s_v[src[x] & 1023];
    }
}

}  // namespace

cudaError_t launch_dec_frame(const int16_t* levels, const uint16_t* ref, const int16_t* mv, const uint8_t* tu_log2,
                             int G, int64_t gstride, int Hp, int Wp, const xv_params* p, int64_t pu_gstride,
                             uint16_t* recon, uint64_t* bits, int64_t bits_gstride, cudaStream_t st) {
    switch (p->ctu) {
        case 8: return dec_n<8>(levels, ref, mv, tu_log2, G, gstride, Hp, Wp, p->qp, pu_gstride, recon, bits, bits_gstride, st);
        case 16: return dec_n<16>(levels, ref, mv, tu_log2, G, gstride, Hp, Wp, p->qp, pu_gstride, recon, bits, bits_gstride, st);
        case 32: return dec_n<32>(levels, ref, mv, tu_log2, G, gstride, Hp, Wp, p->qp, pu_gstride, recon, bits, bits_gstride, st);
        case 64: return dec_n<64>(levels, ref, mv, tu_log2, G, gstride, Hp, Wp, p->qp, pu_gstride, recon, bits, bits_gstride, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_unpack(const uint16_t* recon, int bands, int T, int H, int W, int Hp, int Wp, const double* minmax,
                          float* dst, cudaStream_t st) {
    const int64_t rows = (int64_t)T * H;
    int64_t bx = (rows + (kUnpackThreads / 32) * 4 - 1) / ((kUnpackThreads / 32) * 4);
    if (bx > 1024) bx = 1024;
    dim3 grid((unsigned)(bx < 1 ? 1 : bx), bands);
    k_unpack<<<grid, kUnpackThreads, 0, st>>>(recon, T, H, W, Hp, Wp, minmax, dst);
    return cudaGetLastError();
}

}  // namespace xvh
