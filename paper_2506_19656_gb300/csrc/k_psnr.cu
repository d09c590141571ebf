// k_psnr.cu -- PSNR per band against the original cube (paper Sec. 2.3: the
// peak is the maximum intensity of the original sequence for each channel).
//
// Band b lives in group b/3, channel b%3 of the reconstruction.  Each sample
// is de-quantised as min + q (max - min)/1023 (one double multiply, one
// double add, as in the definition) and compared with the original; the
// exact 10-bit error against the quantised planes is accumulated alongside.
//
// FP64 issue is scarce on this part, so the per-sample loop runs in FP32:
// the 1024 possible de-quantised doubles of the band are tabulated in shared
// memory, each split exactly into three floats (h + l + l2: 24 + 24 + 5
// significant bits); e = x - (h + l + l2) is formed in float-float with
// TwoSum steps, squared with an FMA-exact product and accumulated in
// float-float per thread, and only the thread totals are summed in double.
// The error of a term is about u^2 |e| + u^3 |x^| (u = 2^-24), far below the
// double rounding of the definition itself.  Bands with max(|min|, |max|)
// outside [2^-30, 2^50] take the plain double path: below, float subnormals
// could cost the split its exactness; above, a thread's float sum of squares
// could overflow.
// Per-block partials go to context scratch and are summed in a fixed order
// (Kahan) by a second kernel, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cstdint>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kThreads = 256;

// s + err = a + b exactly (Knuth's TwoSum; explicit roundings so that
// nothing is contracted or reassociated)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// kVec: each lane takes 4 consecutive samples with one 16-byte (float) or
// 8-byte (uint16) load per array; chosen by the host when W % 4 == 0 and the
// source is aligned for it (planes and recon rows always are).
template <typename T, int kVec>
__global__ void __launch_bounds__(kThreads)
k_psnr(const T* __restrict__ src, int bands, int T_, int H, int W, const uint16_t* __restrict__ planes,
       const uint16_t* __restrict__ recon, int Hp, int Wp, const BandQ* __restrict__ bq, PsnrPart* part) {
    const int b = blockIdx.y;
    const int g = b / 3, c = b % 3;
    const BandQ q = bq[b];
    const int64_t n = (int64_t)T_ * H * W;
    const T* p = src + (int64_t)b * n;
    const double mag = fmax(fabs(q.lo), fabs(q.hi));
    const bool ff = mag >= 0x1p-30 && mag <= 0x1p50;  // the FP32 path (see above)
    __shared__ float4 s_xh[1024];  // (h, l, l2, unused) of each 10-bit level's de-quantised value
    for (int v = threadIdx.x; v < 1024; v += kThreads) {
        const double xh = __dadd_rn(q.lo, __dmul_rn((double)v, q.delta));
        const float h = __double2float_rn(xh);
        const double r = xh - (double)h;  // exact
        const float l = __double2float_rn(r);
        const float l2 = __double2float_rn(r - (double)l);  // exact: at most 5 significant bits remain
        s_xh[v] = make_float4(h, l, l2, 0.f);
    }
    __syncthreads();
    double sse = 0.0;
    float acc_hi = 0.f, acc_lo = 0.f;  // float-float running sum of e^2
    unsigned long long sse10 = 0, count = 0;
    // one sample: its 10-bit error and its error against the original
    auto sample = [&](float xf, double xd, int rq, int qv) {
        const int e10 = qv - rq;
        sse10 += (unsigned long long)(e10 * e10);
        if (!isfinite(xf)) return;
        ++count;
        const float4 tv = s_xh[rq & 1023];
        if (ff) {
            // e = xf - h - l - l2 in float-float
            float s1, e1, t1, e2, eh, el;
            two_sum(xf, -tv.x, s1, e1);
            two_sum(e1, -tv.y, t1, e2);
            two_sum(s1, t1, eh, el);
            el = __fadd_rn(el, __fsub_rn(e2, tv.z));
            // e^2 = p + pe + 2 eh el (+ el^2, negligible)
            const float pr = __fmul_rn(eh, eh);
            const float pe = __fmaf_rn(eh, eh, -pr);
            const float qq = __fmaf_rn(__fmul_rn(2.f, eh), el, pe);
            float sh, se;
            two_sum(acc_hi, pr, sh, se);
            acc_lo = __fadd_rn(acc_lo, __fadd_rn(se, qq));
            acc_hi = sh;
        } else {
            const double xh = __dadd_rn(q.lo, __dmul_rn((double)rq, q.delta));
            const double e = __dsub_rn(xd, xh);
            sse = __fma_rn(e, e, sse);
        }
    };
    // one warp per image row, the lanes along x; (frame, row) advance by the
    // warp stride without a division per row
    const int lane = threadIdx.x & 31;
    const int warps = (int)gridDim.x * (kThreads / 32);
    const int64_t rows = (int64_t)T_ * H;
    const int64_t cstride = (int64_t)Hp * Wp;
    const int64_t row0 = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    int t = (int)(row0 / H), y = (int)(row0 - (int64_t)t * H);
    const int dt = warps / H, dy = warps - dt * H;
    for (int64_t row = row0; row < rows; row += warps) {
        const T* xr = p + row * W;
        const int64_t base = (((int64_t)g * T_ + t) * 3 + c) * cstride + (int64_t)y * Wp;
        const uint16_t* rr = recon + base;
        const uint16_t* qr = planes + base;
        if constexpr (kVec == 4) {
            for (int x = 4 * lane; x < W; x += 128) {
                const uint2 r4 = *reinterpret_cast<const uint2*>(rr + x);
                const uint2 q4 = *reinterpret_cast<const uint2*>(qr + x);
                float xv[4];
                if constexpr (sizeof(T) == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(xr + x);
                    xv[0] = v.x; xv[1] = v.y; xv[2] = v.z; xv[3] = v.w;
                } else {
                    const uint2 v = *reinterpret_cast<const uint2*>(xr + x);
                    xv[0] = (float)(v.x & 0xffffu); xv[1] = (float)(v.x >> 16);
                    xv[2] = (float)(v.y & 0xffffu); xv[3] = (float)(v.y >> 16);
                }
                const int rqv[4] = {(int)(r4.x & 0xffffu), (int)(r4.x >> 16), (int)(r4.y & 0xffffu), (int)(r4.y >> 16)};
                const int qvv[4] = {(int)(q4.x & 0xffffu), (int)(q4.x >> 16), (int)(q4.y & 0xffffu), (int)(q4.y >> 16)};
#pragma unroll
                for (int i = 0; i < 4; ++i) sample(xv[i], (double)xv[i], rqv[i], qvv[i]);
            }
        } else {
            for (int x = lane; x < W; x += 32) sample((float)xr[x], (double)xr[x], rr[x], qr[x]);
        }
        t += dt;
        y += dy;
        if (y >= H) { y -= H; ++t; }
    }
    sse += (double)acc_hi + (double)acc_lo;
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

// Per band: the block partials (nblk <= 256) summed in a fixed order, so the
// result does not depend on scheduling: lane l sums partials 8l .. 8l+7 in
// order with Kahan compensation, then the 32 lane sums are combined
// pairwise (lanes l and l + o, o = 16, 8, .., 1) with TwoSum, carrying the
// rounding errors alongside.
__global__ void k_psnr_final(const PsnrPart* part, int nblk, PsnrPart* out) {
    const int b = blockIdx.x;
    const int lane = threadIdx.x;  // 32 threads
    double sum = 0.0, comp = 0.0;
    unsigned long long s10 = 0, cnt = 0;
    for (int k = 8 * lane; k < 8 * lane + 8 && k < nblk; ++k) {
        const PsnrPart r = part[(int64_t)b * nblk + k];
        const double y = r.sse - comp;
        const double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
        s10 += r.sse10;
        cnt += r.count;
    }
    double err = -comp;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double a = sum, bb = __shfl_down_sync(0xffffffffu, sum, o);
        const double e2 = __shfl_down_sync(0xffffffffu, err, o);
        const double s2 = a + bb;                          // TwoSum(a, bb)
        const double bv = s2 - a;
        const double te = (a - (s2 - bv)) + (bb - bv);
        sum = s2;
        err = err + e2 + te;
        s10 += __shfl_down_sync(0xffffffffu, s10, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) out[b] = PsnrPart{sum + err, s10, cnt, 0.0};
}

}  // namespace

// Blocks per band: one per 2048 samples, at most 256, and together at most
// one wave of the blocks resident at once (k_psnr<float, 4>, the variant
// with the most registers), so that no partial second wave runs alone.
int psnr_blocks_per_band(int64_t n, int bands) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_psnr<float, 4>, kThreads, 0) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    int64_t want = (n + kThreads * 8 - 1) / (kThreads * 8);
    const int64_t wave = (int64_t)sms * per / (bands > 0 ? bands : 1);
    if (want > wave) want = wave;
    if (want > 256) want = 256;
    return (int)(want < 1 ? 1 : want);
}

cudaError_t launch_psnr(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* planes,
                        const uint16_t* recon, int Hp, int Wp, const BandQ* bq, PsnrPart* part, int nblk,
                        PsnrPart* out, cudaStream_t st) {
    dim3 grid(nblk, bands);
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    if (dt == XV_F32) {
        const float* s = static_cast<const float*>(src);
        if (W % 4 == 0 && a % 16 == 0) k_psnr<float, 4><<<grid, kThreads, 0, st>>>(s, bands, T, H, W, planes, recon, Hp, Wp, bq, part);
        else k_psnr<float, 1><<<grid, kThreads, 0, st>>>(s, bands, T, H, W, planes, recon, Hp, Wp, bq, part);
    } else {
        const uint16_t* s = static_cast<const uint16_t*>(src);
        if (W % 4 == 0 && a % 8 == 0) k_psnr<uint16_t, 4><<<grid, kThreads, 0, st>>>(s, bands, T, H, W, planes, recon, Hp, Wp, bq, part);
        else k_psnr<uint16_t, 1><<<grid, kThreads, 0, st>>>(s, bands, T, H, W, planes, recon, Hp, Wp, bq, part);
    }
    k_psnr_final<<<bands, 32, 0, st>>>(part, nblk, out);
    return cudaGetLastError();
}

}  // namespace xvh
