// k_quant.cu -- per-band min/max and min-max quantisation with band packing.
//
// Paper Sec. 2.1: bands are packed three to a video, the last group padded
// by repeating its last band, and converted to an N-bit integer video (here
// 10 bit by per-band min-max, see xv_quantize_pack in include/xv.h).
//
// Both kernels are HBM-bound streams.  The quantiser's definition is in IEEE
// double, but double-precision throughput is low on this GPU, so each sample
// is first evaluated in float32; the float result r_f differs from the exact
// value by less than 2^-10 whenever |r_f| <= 2048 (three float roundings of at
// most 2^-24 relative each, on a magnitude <= 2048, plus the rounding of s to
// float), so floor(r_f) is the exact answer unless r_f lies within 2^-10 of
// an integer.  Only those samples (about 0.2%) take the double path, which is
// the definition itself: __dsub_rn, __dmul_rn, __dadd_rn, floor.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned float_order(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_float(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

template <typename T>
__device__ __forceinline__ float load_f(const T* p, int64_t i) { return (float)p[i]; }

__global__ void k_mm_init(unsigned* enc, int bands) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < bands) { enc[2 * b] = 0xffffffffu; enc[2 * b + 1] = 0u; }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_minmax(const T* __restrict__ src, int64_t n, unsigned* enc) {
    const int b = blockIdx.y;
    const T* p = src + (int64_t)b * n;
    float lo = FLT_MAX, hi = -FLT_MAX;
    bool any = false;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    // vector part: 8 samples per step when the band start is 16-byte aligned
    constexpr int V = 16 / sizeof(T);
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const int64_t nv = n / V;
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nv; i += stride) {
            uint4 w = __ldg(reinterpret_cast<const uint4*>(p) + i);
            const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                float v = (float)e[k];
                if (isfinite(v)) { lo = fminf(lo, v); hi = fmaxf(hi, v); any = true; }
            }
        }
        done = nv * V;
    }
    for (int64_t i = done + (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        float v = load_f(p, i);
        if (isfinite(v)) { lo = fminf(lo, v); hi = fmaxf(hi, v); any = true; }
    }
    unsigned elo = any ? float_order(lo) : 0xffffffffu, ehi = any ? float_order(hi) : 0u;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        elo = min(elo, __shfl_xor_sync(0xffffffffu, elo, o));
        ehi = max(ehi, __shfl_xor_sync(0xffffffffu, ehi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (elo != 0xffffffffu) atomicMin(&enc[2 * b], elo);
        if (ehi != 0u) atomicMax(&enc[2 * b + 1], ehi);
    }
}

__device__ void fill_bandq(double lo, double hi, BandQ* q) {
    q->lo = lo;
    q->hi = hi;
    q->s = hi > lo ? 1023.0 / (hi - lo) : 0.0;  // IEEE division (correctly rounded)
    q->delta = (hi - lo) / 1023.0;
    q->lo_f = (float)lo;
    q->s_f = (float)q->s;
    q->fast_ok = ((double)q->lo_f == lo) && q->s <= 1e30;
    q->pad = 0;
}

__global__ void k_mm_final(const unsigned* enc, int bands, double* minmax, BandQ* bq) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= bands) return;
    unsigned elo = enc[2 * b], ehi = enc[2 * b + 1];
    double lo = 0.0, hi = 0.0;
    if (elo != 0xffffffffu) {  // at least one finite sample
        lo = (double)order_float(elo);
        hi = (double)order_float(ehi);
    }
    minmax[2 * b] = lo;
    minmax[2 * b + 1] = hi;
    fill_bandq(lo, hi, &bq[b]);
}

__global__ void k_bandq(const double* minmax, int bands, BandQ* bq) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < bands) fill_bandq(minmax[2 * b], minmax[2 * b + 1], &bq[b]);
}

__device__ __forceinline__ int quantize_sample(float x, const BandQ& q) {
    if (!isfinite(x)) return 0;
    if (q.fast_ok) {
        float d = __fsub_rn(x, q.lo_f);
        float p = __fmul_rn(d, q.s_f);
        float r = __fadd_rn(p, 0.5f);
        if (r >= -1.0f && r <= 2048.0f) {
            float k = floorf(r);
            const float eps = 0.0009765625f;  // 2^-10
            if (r - k >= eps && (k + 1.0f) - r >= eps) {
                int ki = (int)k;
                return ki < 0 ? 0 : (ki > 1023 ? 1023 : ki);
            }
        }
    }
    double d = __dsub_rn((double)x, q.lo);
    double p = __dmul_rn(d, q.s);
    double r = __dadd_rn(p, 0.5);
    double f = floor(r);
    if (f < 0.0) return 0;
    if (f > 1023.0) return 1023;
    return (int)f;
}

// Mixed-radix position of an item: (g, t, c, y, xv) with item index
// (((g T + t) 3 + c) Hp + y) wv + xv.
struct QPos {
    int64_t g;
    int t, c, y, xv;
};

__device__ __forceinline__ QPos qpos(int64_t it, int wv, int Hp, int T_) {
    QPos p;
    const int64_t row = it / wv;
    p.xv = (int)(it - row * wv);
    const int64_t f = row / Hp;
    p.y = (int)(row - f * Hp);
    const int64_t gt = f / 3;
    p.c = (int)(f - gt * 3);
    p.g = gt / T_;
    p.t = (int)(gt - p.g * T_);
    return p;
}

// One thread: 8 consecutive output samples of one plane row.  The grid
// stride's position is added to the item's position digit by digit with
// carries, so the loop divides only once.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_quant_pack(const T* __restrict__ src, int bands, int T_, int H, int W, int Hp, int Wp,
             const BandQ* __restrict__ bq, uint16_t* __restrict__ planes, int64_t items) {
    const int wv = Wp / 8;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t it = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    QPos p = qpos(it, wv, Hp, T_);
    const QPos d = qpos(stride, wv, Hp, T_);
    for (; it < items; it += stride) {
        const int xv = p.xv, y = p.y, c = p.c, t = p.t;
        const int64_t row = ((p.g * T_ + t) * 3 + c) * Hp + y;
        int b = (int)(3 * p.g + c);
        if (b >= bands) b = bands - 1;
        const BandQ q = bq[b];
        const int sy = y < H ? y : H - 1;
        const T* srow = src + (((int64_t)b * T_ + t) * H + sy) * W;
        const int x0 = xv * 8;
        float v[8];
        if (x0 + 8 <= W && (reinterpret_cast<uintptr_t>(srow + x0) & 15) == 0) {
            if constexpr (sizeof(T) == 4) {
                float4 a = __ldg(reinterpret_cast<const float4*>(srow + x0));
                float4 e = __ldg(reinterpret_cast<const float4*>(srow + x0) + 1);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = e.x; v[5] = e.y; v[6] = e.z; v[7] = e.w;
            } else {
                uint4 w = __ldg(reinterpret_cast<const uint4*>(srow + x0));
                const uint16_t* h = reinterpret_cast<const uint16_t*>(&w);
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = (float)h[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int sx = x0 + k < W ? x0 + k : W - 1;
                v[k] = (float)srow[sx];
            }
        }
        uint4 out;
        uint16_t* o = reinterpret_cast<uint16_t*>(&out);
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = (uint16_t)quantize_sample(v[k], q);
        *reinterpret_cast<uint4*>(planes + row * Wp + x0) = out;
        // advance the position by the stride
        int carry;
        p.xv += d.xv; carry = p.xv >= wv; if (carry) p.xv -= wv;
        p.y += d.y + carry; carry = p.y >= Hp; if (carry) p.y -= Hp;
        p.c += d.c + carry; carry = p.c >= 3; if (carry) p.c -= 3;
        p.t += d.t + carry; carry = p.t >= T_; if (carry) p.t -= T_;
        p.g += d.g + carry;
    }
}

// Grid of a grid-stride kernel over `items` threads' work: at most one full
// wave of the blocks that are resident at once (a second, partial wave would
// leave most of the GPU idle while it runs).
template <typename K>
int grid_for(K kernel, int64_t items) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, 0) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    const int64_t want = (items + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sms * per;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_minmax(const void* src, xv_dtype dt, int bands, int64_t n, unsigned* enc, double* minmax,
                          BandQ* bq, cudaStream_t st) {
    k_mm_init<<<(bands + 31) / 32, 32, 0, st>>>(enc, bands);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_band = (int)((int64_t)sms * 8 / bands);
    if (per_band < 1) per_band = 1;
    int64_t need = (n / 8 + kThreads - 1) / kThreads;
    if (per_band > need) per_band = (int)(need > 0 ? need : 1);
    dim3 grid(per_band, bands);
    if (dt == XV_F32)
        k_minmax<float><<<grid, kThreads, 0, st>>>(static_cast<const float*>(src), n, enc);
    else
        k_minmax<uint16_t><<<grid, kThreads, 0, st>>>(static_cast<const uint16_t*>(src), n, enc);
    k_mm_final<<<(bands + 31) / 32, 32, 0, st>>>(enc, bands, minmax, bq);
    return cudaGetLastError();
}

cudaError_t launch_prepare_bands(const void* src, xv_dtype dt, int bands, int64_t n, double* minmax, int fixed,
                                 unsigned* enc, BandQ* bq, cudaStream_t st) {
    if (fixed) return launch_bandq(minmax, bands, bq, st);
    return launch_minmax(src, dt, bands, n, enc, minmax, bq, st);
}

cudaError_t launch_bandq(const double* minmax, int bands, BandQ* bq, cudaStream_t st) {
    k_bandq<<<(bands + 31) / 32, 32, 0, st>>>(minmax, bands, bq);
    return cudaGetLastError();
}

cudaError_t launch_quantize_pack(const void* src, xv_dtype dt, int bands, int T, int H, int W, int Hp, int Wp,
                                 const BandQ* bq, uint16_t* planes, cudaStream_t st) {
    const int G = (bands + 2) / 3;
    const int64_t items = (int64_t)G * T * 3 * Hp * (Wp / 8);
    if (items == 0) return cudaSuccess;
    if (dt == XV_F32)
        k_quant_pack<float><<<grid_for(k_quant_pack<float>, items), kThreads, 0, st>>>(
            static_cast<const float*>(src), bands, T, H, W, Hp, Wp, bq, planes, items);
    else
        k_quant_pack<uint16_t><<<grid_for(k_quant_pack<uint16_t>, items), kThreads, 0, st>>>(
            static_cast<const uint16_t*>(src), bands, T, H, W, Hp, Wp, bq, planes, items);
    return cudaGetLastError();
}

}  // namespace xvh
