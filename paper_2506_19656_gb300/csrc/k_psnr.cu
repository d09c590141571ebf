// k_psnr.cu -- PSNR per band against the original cube (paper Sec. 2.3: the
// peak is the maximum intensity of the original sequence for each channel).
//
// Band b lives in group b/3, channel b%3 of the reconstruction.  Each sample
// is de-quantised as min + q (max - min)/1023 (one double multiply, one
// double add, as in the definition) and compared with the original; the
// exact 10-bit error against the quantised planes is accumulated alongside.
// Per-block partials go to context scratch and are summed in a fixed order
// (Kahan) by a second kernel, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cstdint>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_psnr(const T* __restrict__ src, int bands, int T_, int H, int W, const uint16_t* __restrict__ planes,
       const uint16_t* __restrict__ recon, int Hp, int Wp, const BandQ* __restrict__ bq, PsnrPart* part) {
    const int b = blockIdx.y;
    const int g = b / 3, c = b % 3;
    const BandQ q = bq[b];
    const int64_t n = (int64_t)T_ * H * W;
    (void)n;
    const T* p = src + (int64_t)b * n;
    double sse = 0.0;
    unsigned long long sse10 = 0, count = 0;
    // one warp per image row: the row's frame and y are derived once, the
    // lanes stride along x
    const int lane = threadIdx.x & 31;
    const int warps = (int)gridDim.x * (kThreads / 32);
    const int64_t rows = (int64_t)T_ * H;
    const int64_t cstride = (int64_t)Hp * Wp;
    for (int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); row < rows; row += warps) {
        const int t = (int)(row / H), y = (int)(row - (int64_t)t * H);
        const T* xr = p + row * W;
        const int64_t base = (((int64_t)g * T_ + t) * 3 + c) * cstride + (int64_t)y * Wp;
        const uint16_t* rr = recon + base;
        const uint16_t* qr = planes + base;
        for (int x = lane; x < W; x += 32) {
            const int rq = rr[x];
            const int e10 = (int)qr[x] - rq;
            sse10 += (unsigned long long)(e10 * e10);
            const double xv = (double)xr[x];
            if (isfinite(xv)) {
                const double xh = __dadd_rn(q.lo, __dmul_rn((double)rq, q.delta));
                const double e = __dsub_rn(xv, xh);
                sse = __dadd_rn(sse, __dmul_rn(e, e));
                ++count;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sse += __shfl_xor_sync(0xffffffffu, sse, o);
        sse10 += __shfl_xor_sync(0xffffffffu, sse10, o);
        count += __shfl_xor_sync(0xffffffffu, count, o);
    }
    __shared__ double s_sse[kThreads / 32];
    __shared__ unsigned long long s_10[kThreads / 32], s_n[kThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_sse[w] = sse; s_10[w] = sse10; s_n[w] = count; }
    __syncthreads();
    if (threadIdx.x == 0) {
        PsnrPart r{0.0, 0ull, 0ull, 0.0};
        for (int k = 0; k < kThreads / 32; ++k) { r.sse += s_sse[k]; r.sse10 += s_10[k]; r.count += s_n[k]; }
        part[(int64_t)b * gridDim.x + blockIdx.x] = r;
    }
}

__global__ void k_psnr_final(const PsnrPart* part, int nblk, PsnrPart* out) {
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    double sum = 0.0, comp = 0.0;
    unsigned long long s10 = 0, cnt = 0;
    for (int k = 0; k < nblk; ++k) {
        const PsnrPart& r = part[(int64_t)b * nblk + k];
        double y = r.sse - comp;  // Kahan summation in block order
        double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
        s10 += r.sse10;
        cnt += r.count;
    }
    out[b] = PsnrPart{sum, s10, cnt, 0.0};
}

}  // namespace

int psnr_blocks_per_band(int64_t n) {
    int64_t want = (n + kThreads * 8 - 1) / (kThreads * 8);
    if (want > 256) want = 256;
    return (int)(want < 1 ? 1 : want);
}

cudaError_t launch_psnr(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* planes,
                        const uint16_t* recon, int Hp, int Wp, const BandQ* bq, PsnrPart* part, int nblk,
                        PsnrPart* out, cudaStream_t st) {
    dim3 grid(nblk, bands);
    if (dt == XV_F32)
        k_psnr<float><<<grid, kThreads, 0, st>>>(static_cast<const float*>(src), bands, T, H, W, planes, recon,
                                                  Hp, Wp, bq, part);
    else
        k_psnr<uint16_t><<<grid, kThreads, 0, st>>>(static_cast<const uint16_t*>(src), bands, T, H, W, planes,
                                                     recon, Hp, Wp, bq, part);
    k_psnr_final<<<bands, 32, 0, st>>>(part, nblk, out);
    return cudaGetLastError();
}

}  // namespace xvh
