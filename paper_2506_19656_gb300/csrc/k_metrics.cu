// k_metrics.cu -- SSIM per band and the mean spectral angle between a cube
// and its reconstruction (the paper's other two quality metrics, Sec. 2.3),
// with the definitions of xv_ssim and xv_sa in include/xv.h.
//
// SSIM runs in FP32 on band-normalised data x' = (x - min) / L (L = max -
// min), every value in [0, 1].  The contrast-structure factor
// (2 s_xy + C2) / (s_x^2 + s_y^2 + C2) is unchanged by the shift and the
// scale (C2 scales with L^2); the luminance factor compares absolute means
// m = min / L + mu' and is evaluated through the identity
// 2 m_x m_y + C1 = (m_x^2 + m_y^2 + C1) - (m_x - m_y)^2, i.e.
// 1 - (mu'_x - mu'_y)^2 / (m_x^2 + m_y^2 + C1), where the difference comes
// from the shifted means (no cancellation however large the offset).  A
// block takes a tile of 32 x 32 window positions of one frame: the Gaussian
// means by a separable pass through shared memory, then the variances and
// the covariance directly over each 11 x 11 window (deviations from the
// local mean, so nothing cancels), each thread taking four vertically
// adjacent windows so that every sample load serves up to four of them.  The spectral angle takes the
// per-band differences d = x^ - x in double, the wedge terms
// s_i d_j - s_j d_i (= s_i s^_j - s_j s^_i) and the dot product in FP32, and
// atan2.  Per-block partials are summed in a fixed order by a final kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kSsimTX = 32, kSsimTY = 32;                  // window positions per tile
constexpr int kSsimIX = kSsimTX + 10, kSsimIY = kSsimTY + 10;  // input tile
constexpr int kSsimThreads = 256;
constexpr int kSsimRows = 4;  // vertically adjacent windows per thread (they share sample loads)

struct Gauss11 {
    float w[11];
    float w2[121];  // w[u] w[v]: kernel parameters are free FMA operands
};

template <typename T>
__global__ void __launch_bounds__(kSsimThreads)
k_ssim(const T* __restrict__ src, int T_, int H, int W, const uint16_t* __restrict__ recon, int Hp, int Wp,
       const BandQ* __restrict__ bq, Gauss11 g, MetricPart* part) {
    const int b = blockIdx.y, grp = b / 3, ch = b % 3;
    const BandQ q = bq[b];
    const int tid = threadIdx.x;
    __shared__ float s_x[kSsimIY][kSsimIX], s_y[kSsimIY][kSsimIX];
    __shared__ float s_hx[kSsimIY][kSsimTX], s_hy[kSsimIY][kSsimTX];
    __shared__ float s_mx[kSsimTY][kSsimTX], s_my[kSsimTY][kSsimTX];
    __shared__ unsigned char s_bad[kSsimIY][kSsimIX];
    __shared__ unsigned char s_hbad[kSsimIY][kSsimTX];
    __shared__ float s_yv[1024];  // normalised de-quantised value of each level
    __shared__ double s_sum[kSsimThreads / 32];
    __shared__ unsigned long long s_n[kSsimThreads / 32];
    const double L = q.hi - q.lo;
    double sum = 0.0;
    unsigned long long n = 0;
    if (L > 0.0) {
        for (int v = tid; v < 1024; v += kSsimThreads)
            s_yv[v] = (float)((__dadd_rn(q.lo, __dmul_rn((double)v, q.delta)) - q.lo) / L);
        const float lo_f = (float)q.lo, inv_l = (float)(1.0 / L), off = (float)(q.lo / L);
        const float C1 = 1e-4f, C2 = 9e-4f;  // (0.01)^2, (0.03)^2 on normalised data
        const int ox_n = W - 10, oy_n = H - 10;  // window positions per row / column
        const int tx_n = (ox_n + kSsimTX - 1) / kSsimTX, ty_n = (oy_n + kSsimTY - 1) / kSsimTY;
        const int64_t tiles = (int64_t)T_ * ty_n * tx_n;
        const int64_t n_src = (int64_t)T_ * H * W;
        for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            const int t = (int)(tile / ((int64_t)ty_n * tx_n));
            const int rem = (int)(tile - (int64_t)t * ty_n * tx_n);
            const int y0 = (rem / tx_n) * kSsimTY, x0 = (rem % tx_n) * kSsimTX;
            const T* xs = src + (int64_t)b * n_src + (int64_t)t * H * W;
            const uint16_t* rs = recon + (((int64_t)grp * T_ + t) * 3 + ch) * Hp * Wp;
            __syncthreads();  // the previous tile's shared data is no longer read
            for (int i = tid; i < kSsimIY * kSsimIX; i += kSsimThreads) {
                const int r = i / kSsimIX, c = i - r * kSsimIX;
                const int yy = min(y0 + r, H - 1), xx = min(x0 + c, W - 1);  // past the edge: unused positions
                const float xv = (float)xs[(int64_t)yy * W + xx];
                const bool ok = isfinite(xv);
                s_x[r][c] = ok ? (xv - lo_f) * inv_l : 0.f;
                s_bad[r][c] = ok ? 0 : 1;
                s_y[r][c] = s_yv[rs[(int64_t)yy * Wp + xx] & 1023];
            }
            __syncthreads();
            for (int i = tid; i < kSsimIY * kSsimTX; i += kSsimThreads) {
                const int r = i / kSsimTX, c = i - r * kSsimTX;
                float ax = 0.f, ay = 0.f;
                unsigned char bad = 0;
#pragma unroll
                for (int v = 0; v < 11; ++v) {
                    ax = fmaf(g.w[v], s_x[r][c + v], ax);
                    ay = fmaf(g.w[v], s_y[r][c + v], ay);
                    bad |= s_bad[r][c + v];
                }
                s_hx[r][c] = ax;
                s_hy[r][c] = ay;
                s_hbad[r][c] = bad;
            }
            __syncthreads();
            for (int i = tid; i < kSsimTY * kSsimTX; i += kSsimThreads) {
                const int r = i / kSsimTX, c = i - r * kSsimTX;
                float ax = 0.f, ay = 0.f;
#pragma unroll
                for (int u = 0; u < 11; ++u) {
                    ax = fmaf(g.w[u], s_hx[r + u][c], ax);
                    ay = fmaf(g.w[u], s_hy[r + u][c], ay);
                }
                s_mx[r][c] = ax;
                s_my[r][c] = ay;
            }
            __syncthreads();
            {
                // thread: column c, windows r0 .. r0 + 3; every sample of the 14
                // input rows is loaded once and used by the windows covering it
                const int c = tid % kSsimTX, r0 = (tid / kSsimTX) * kSsimRows;
                float mx[kSsimRows], my[kSsimRows], sxx[kSsimRows], syy[kSsimRows], sxy[kSsimRows];
#pragma unroll
                for (int j = 0; j < kSsimRows; ++j) {
                    mx[j] = s_mx[r0 + j][c];
                    my[j] = s_my[r0 + j][c];
                    sxx[j] = syy[j] = sxy[j] = 0.f;
                }
#pragma unroll
                for (int k = 0; k < 10 + kSsimRows; ++k) {
#pragma unroll
                    for (int v = 0; v < 11; ++v) {
                        const float x = s_x[r0 + k][c + v], y = s_y[r0 + k][c + v];
#pragma unroll
                        for (int j = 0; j < kSsimRows; ++j) {
                            const int u = k - j;
                            if (u < 0 || u > 10) continue;  // resolved at compile time
                            const float dx = x - mx[j], dy = y - my[j];
                            const float wdx = g.w2[u * 11 + v] * dx;
                            sxx[j] = fmaf(wdx, dx, sxx[j]);
                            sxy[j] = fmaf(wdx, dy, sxy[j]);
                            syy[j] = fmaf(g.w2[u * 11 + v] * dy, dy, syy[j]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < kSsimRows; ++j) {
                    const int r = r0 + j;
                    if (y0 + r >= oy_n || x0 + c >= ox_n) continue;
                    unsigned char bad = 0;
#pragma unroll
                    for (int u = 0; u < 11; ++u) bad |= s_hbad[r + u][c];
                    if (bad) continue;
                    const float ax = off + mx[j], ay = off + my[j], dm = mx[j] - my[j];
                    const float lum = 1.f - dm * dm / (ax * ax + ay * ay + C1);
                    sum += (double)(lum * (2.f * sxy[j] + C2) / (sxx[j] + syy[j] + C2));
                    ++n;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if ((tid & 31) == 0) { s_sum[tid >> 5] = sum; s_n[tid >> 5] = n; }
    __syncthreads();
    if (tid == 0) {
        MetricPart r{0.0, 0ull};
        for (int k = 0; k < kSsimThreads / 32; ++k) { r.sum += s_sum[k]; r.n += s_n[k]; }
        part[(int64_t)b * gridDim.x + blockIdx.x] = r;
    }
}

constexpr int kSaThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kSaThreads)
k_sa(const T* __restrict__ src, int bands, int T_, int H, int W, const uint16_t* __restrict__ recon, int Hp, int Wp,
     const BandQ* __restrict__ bq, MetricPart* part) {
    __shared__ BandQ s_q[XV_MAX_BANDS];
    __shared__ double s_sum[kSaThreads / 32];
    __shared__ unsigned long long s_n[kSaThreads / 32];
    if (threadIdx.x < bands) s_q[threadIdx.x] = bq[threadIdx.x];
    __syncthreads();
    const int64_t npix = (int64_t)T_ * H * W, n_src = npix;
    double sum = 0.0;
    unsigned long long n = 0;
    for (int64_t p = (int64_t)blockIdx.x * kSaThreads + threadIdx.x; p < npix; p += (int64_t)gridDim.x * kSaThreads) {
        const int t = (int)(p / ((int64_t)H * W));
        const int rem = (int)(p - (int64_t)t * H * W), y = rem / W, x = rem - y * W;
        float s[XV_MAX_BANDS], d[XV_MAX_BANDS];
        bool ok = true;
        float n1 = 0.f, n2 = 0.f, dot = 0.f;
        for (int b = 0; b < bands; ++b) {
            const int grp = b / 3, ch = b % 3;
            const float sv = (float)src[(int64_t)b * n_src + p];
            const int qv = recon[((((int64_t)grp * T_ + t) * 3 + ch) * Hp + y) * Wp + x];
            const double xh = __dadd_rn(s_q[b].lo, __dmul_rn((double)qv, s_q[b].delta));
            const float dv = (float)(xh - (double)sv);
            ok = ok && isfinite(sv);
            s[b] = sv;
            d[b] = dv;
            const float sh = sv + dv;
            n1 = fmaf(sv, sv, n1);
            n2 = fmaf(sh, sh, n2);
            dot = fmaf(sv, sh, dot);
        }
        if (!ok || !(n1 > 0.f) || !(n2 > 0.f)) continue;
        float cr = 0.f;
        for (int i = 0; i < bands; ++i)
            for (int j = i + 1; j < bands; ++j) {
                const float m = fmaf(s[i], d[j], -s[j] * d[i]);
                cr = fmaf(m, m, cr);
            }
        sum += (double)atan2f(sqrtf(cr), dot);
        ++n;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if ((threadIdx.x & 31) == 0) { s_sum[threadIdx.x >> 5] = sum; s_n[threadIdx.x >> 5] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        MetricPart r{0.0, 0ull};
        for (int k = 0; k < kSaThreads / 32; ++k) { r.sum += s_sum[k]; r.n += s_n[k]; }
        part[blockIdx.x] = r;
    }
}

// Per row of partials (one per band, or one for the angle): the sum in a
// fixed order (32 in-order Kahan sums, then a fixed pairwise tree).
__global__ void k_metric_final(const MetricPart* part, int nblk, MetricPart* out) {
    const int b = blockIdx.x, lane = threadIdx.x;
    const int per = (nblk + 31) / 32;
    double sum = 0.0, comp = 0.0;
    unsigned long long cnt = 0;
    for (int k = per * lane; k < per * lane + per && k < nblk; ++k) {
        const MetricPart r = part[(int64_t)b * nblk + k];
        const double y = r.sum - comp;
        const double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
        cnt += r.n;
    }
    double err = -comp;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double a = sum, bb = __shfl_down_sync(0xffffffffu, sum, o);
        const double e2 = __shfl_down_sync(0xffffffffu, err, o);
        const double s2 = a + bb;
        const double bv = s2 - a;
        const double te = (a - (s2 - bv)) + (bb - bv);
        sum = s2;
        err = err + e2 + te;
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) out[b] = MetricPart{sum + err, cnt};
}

}  // namespace

int ssim_blocks_per_band(int T, int H, int W) {
    if (H < 11 || W < 11) return 1;
    const int64_t tiles = (int64_t)T * ((H - 10 + kSsimTY - 1) / kSsimTY) * ((W - 10 + kSsimTX - 1) / kSsimTX);
    return (int)(tiles < 512 ? (tiles < 1 ? 1 : tiles) : 512);
}

int sa_blocks(int64_t npix) {
    const int64_t want = (npix + kSaThreads * 4 - 1) / (kSaThreads * 4);
    return (int)(want < 1 ? 1 : (want > 1024 ? 1024 : want));
}

cudaError_t launch_ssim(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* recon, int Hp,
                        int Wp, const BandQ* bq, MetricPart* part, int nblk, MetricPart* out, cudaStream_t st) {
    Gauss11 g;
    double w[11], s = 0.0;
    for (int k = 0; k < 11; ++k) {
        w[k] = std::exp(-(double)((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5));
        s += w[k];
    }
    for (int k = 0; k < 11; ++k) g.w[k] = (float)(w[k] / s);
    for (int u = 0; u < 11; ++u)
        for (int v = 0; v < 11; ++v) g.w2[u * 11 + v] = (float)((w[u] / s) * (w[v] / s));
    dim3 grid(nblk, bands);
    if (H >= 11 && W >= 11) {
        if (dt == XV_F32)
            k_ssim<float><<<grid, kSsimThreads, 0, st>>>(static_cast<const float*>(src), T, H, W, recon, Hp, Wp, bq, g, part);
        else
            k_ssim<uint16_t><<<grid, kSsimThreads, 0, st>>>(static_cast<const uint16_t*>(src), T, H, W, recon, Hp, Wp,
                                                            bq, g, part);
    } else {
        cudaMemsetAsync(part, 0, sizeof(MetricPart) * (size_t)nblk * bands, st);
    }
    k_metric_final<<<bands, 32, 0, st>>>(part, nblk, out);
    return cudaGetLastError();
}

cudaError_t launch_sa(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* recon, int Hp,
                      int Wp, const BandQ* bq, MetricPart* part, int nblk, MetricPart* out, cudaStream_t st) {
    if (dt == XV_F32)
        k_sa<float><<<nblk, kSaThreads, 0, st>>>(static_cast<const float*>(src), bands, T, H, W, recon, Hp, Wp, bq, part);
    else
        k_sa<uint16_t><<<nblk, kSaThreads, 0, st>>>(static_cast<const uint16_t*>(src), bands, T, H, W, recon, Hp, Wp,
                                                    bq, part);
    k_metric_final<<<1, 32, 0, st>>>(part, nblk, out);
    return cudaGetLastError();
}

}  // namespace xvh
