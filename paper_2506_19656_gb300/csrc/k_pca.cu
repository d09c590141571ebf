// k_pca.cu -- PCA over the bands of a cube (the paper's optional transform
// before packing, Sec. 2.1): the fit (band means, then the covariance of the
// centred values), the eigen-decomposition on the host (cyclic Jacobi, the
// matrix is at most 16 x 16), and the per-pixel projection and inverse.
// Definitions: xv_pca_fit / xv_pca_project / xv_pca_inverse in include/xv.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kPcaThreads = 256;
constexpr int kMaxB = XV_MAX_BANDS;

// Pass 1: per block, the sums of every band over the pixels whose bands are
// all finite, and their count.  part: [nblk][kMaxB + 1] doubles (the last:
// the count).
template <typename T>
__global__ void __launch_bounds__(kPcaThreads)
k_pca_sums(const T* __restrict__ src, int bands, int64_t npix, double* part) {
    double acc[kMaxB];
#pragma unroll
    for (int b = 0; b < kMaxB; ++b) acc[b] = 0.0;
    double cnt = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * kPcaThreads + threadIdx.x; p < npix; p += (int64_t)gridDim.x * kPcaThreads) {
        float v[kMaxB];
        bool ok = true;
#pragma unroll
        for (int b = 0; b < kMaxB; ++b) {
            v[b] = b < bands ? (float)src[(int64_t)b * npix + p] : 0.f;
            ok = ok && isfinite(v[b]);
        }
        if (!ok) continue;
#pragma unroll
        for (int b = 0; b < kMaxB; ++b) acc[b] += (double)v[b];
        cnt += 1.0;
    }
    __shared__ double s_red[kPcaThreads / 32][kMaxB + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int b = 0; b <= kMaxB; ++b) {
        double x = b < kMaxB ? acc[b] : cnt;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[w][b] = x;
    }
    __syncthreads();
    if (threadIdx.x <= kMaxB) {
        double x = 0.0;
        for (int k = 0; k < kPcaThreads / 32; ++k) x += s_red[k][threadIdx.x];
        part[(int64_t)blockIdx.x * (kMaxB + 1) + threadIdx.x] = x;
    }
}

struct PcaMean {
    double m[kMaxB];
};

// Pass 2: per block, sum over valid pixels of c_i c_j (c = x - mean) for
// i <= j: a tile of 256 pixels' centred values (double) in shared memory;
// each pair is summed by 256 / npair threads over interleaved pixels (all
// threads busy however few the bands), the parts combined in a fixed order
// at the end.  The covariance is the accurate part of the fit: the smallest
// principal components sit in tiny eigenvalue gaps.  part: [nblk][136].
template <typename T>
__global__ void __launch_bounds__(kPcaThreads)
k_pca_cov(const T* __restrict__ src, int bands, int64_t npix, PcaMean mean, double* part) {
    __shared__ double s_c[kMaxB][kPcaThreads];
    const int npair = bands * (bands + 1) / 2;
    const int nsplit = kPcaThreads / npair;  // threads per pair
    const int pr = (int)threadIdx.x % npair, part_of = (int)threadIdx.x / npair;
    const bool active = part_of < nsplit;
    int pi = 0, pj = 0;
    {  // pair index -> (i, j), i <= j, row by row
        int k = pr;
        while (k >= bands - pi) { k -= bands - pi; ++pi; }
        pj = pi + k;
    }
    double acc = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * kPcaThreads; base < npix; base += (int64_t)gridDim.x * kPcaThreads) {
        const int64_t p = base + threadIdx.x;
        double v[kMaxB];
        bool ok = p < npix;
#pragma unroll
        for (int b = 0; b < kMaxB; ++b) {
            v[b] = (ok && b < bands) ? (double)src[(int64_t)b * npix + p] - mean.m[b] : 0.0;
            ok = ok && isfinite(v[b]);
        }
        __syncthreads();  // the previous tile is no longer read
#pragma unroll
        for (int b = 0; b < kMaxB; ++b) s_c[b][threadIdx.x] = ok ? v[b] : 0.0;
        __syncthreads();
        if (active)
            for (int q = part_of; q < kPcaThreads; q += nsplit) acc = fma(s_c[pi][q], s_c[pj][q], acc);
    }
    // combine the parts of each pair in part order
    __syncthreads();
    double* s_acc = &s_c[0][0];  // kMaxB * 256 doubles >= 256 partial sums
    s_acc[threadIdx.x] = active ? acc : 0.0;
    __syncthreads();
    if ((int)threadIdx.x < npair) {
        double t = 0.0;
        for (int k = 0; k < nsplit; ++k) t += s_acc[k * npair + threadIdx.x];
        part[(int64_t)blockIdx.x * 136 + threadIdx.x] = t;
    }
}

struct PcaBasis {
    float m[kMaxB];
    float v[kMaxB][kMaxB];  // [component][band]
};

// 4 consecutive pixels of one band (16-byte float or 8-byte uint16 load).
template <typename T>
__device__ __forceinline__ float4 load4(const T* p) {
    if constexpr (sizeof(T) == 4) {
        return *reinterpret_cast<const float4*>(p);
    } else {
        const uint2 w = *reinterpret_cast<const uint2*>(p);
        return make_float4((float)(w.x & 0xffffu), (float)(w.x >> 16), (float)(w.y & 0xffffu), (float)(w.y >> 16));
    }
}

// kVec: 4 pixels per thread with vector loads and stores (npix % 4 == 0 and
// aligned arrays, chosen by the host), else one.
template <typename T, int kVec>
__global__ void __launch_bounds__(kPcaThreads)
k_pca_project(const T* __restrict__ src, int bands, int npc, int64_t npix, PcaBasis B, float* __restrict__ dst) {
    const int64_t nq = npix / kVec;
    for (int64_t q = (int64_t)blockIdx.x * kPcaThreads + threadIdx.x; q < nq; q += (int64_t)gridDim.x * kPcaThreads) {
        const int64_t p = q * kVec;
        float c[kMaxB][kVec];
#pragma unroll
        for (int b = 0; b < kMaxB; ++b) {
            if (b < bands) {
                if constexpr (kVec == 4) {
                    const float4 v = load4(src + (int64_t)b * npix + p);
                    c[b][0] = v.x - B.m[b]; c[b][1] = v.y - B.m[b]; c[b][2] = v.z - B.m[b]; c[b][3] = v.w - B.m[b];
                } else {
                    c[b][0] = (float)src[(int64_t)b * npix + p] - B.m[b];
                }
            } else {
#pragma unroll
                for (int e = 0; e < kVec; ++e) c[b][e] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxB; ++k) {
            if (k >= npc) break;
            float z[kVec];
#pragma unroll
            for (int e = 0; e < kVec; ++e) z[e] = 0.f;
#pragma unroll
            for (int b = 0; b < kMaxB; ++b)
                if (b < bands)
#pragma unroll
                    for (int e = 0; e < kVec; ++e) z[e] = fmaf(B.v[k][b], c[b][e], z[e]);
            if constexpr (kVec == 4) *reinterpret_cast<float4*>(dst + (int64_t)k * npix + p) = make_float4(z[0], z[1], z[2], z[3]);
            else dst[(int64_t)k * npix + p] = z[0];
        }
    }
}

template <int kVec>
__global__ void __launch_bounds__(kPcaThreads)
k_pca_inverse(const float* __restrict__ z, int npc, int bands, int64_t npix, PcaBasis B, float* __restrict__ dst) {
    const int64_t nq = npix / kVec;
    for (int64_t q = (int64_t)blockIdx.x * kPcaThreads + threadIdx.x; q < nq; q += (int64_t)gridDim.x * kPcaThreads) {
        const int64_t p = q * kVec;
        float zz[kMaxB][kVec];
#pragma unroll
        for (int k = 0; k < kMaxB; ++k) {
            if (k < npc) {
                if constexpr (kVec == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(z + (int64_t)k * npix + p);
                    zz[k][0] = v.x; zz[k][1] = v.y; zz[k][2] = v.z; zz[k][3] = v.w;
                } else {
                    zz[k][0] = z[(int64_t)k * npix + p];
                }
            } else {
#pragma unroll
                for (int e = 0; e < kVec; ++e) zz[k][e] = 0.f;
            }
        }
#pragma unroll
        for (int b = 0; b < kMaxB; ++b) {
            if (b >= bands) break;
            float x[kVec];
#pragma unroll
            for (int e = 0; e < kVec; ++e) x[e] = B.m[b];
#pragma unroll
            for (int k = 0; k < kMaxB; ++k)
                if (k < npc)
#pragma unroll
                    for (int e = 0; e < kVec; ++e) x[e] = fmaf(B.v[k][b], zz[k][e], x[e]);
            if constexpr (kVec == 4) *reinterpret_cast<float4*>(dst + (int64_t)b * npix + p) = make_float4(x[0], x[1], x[2], x[3]);
            else dst[(int64_t)b * npix + p] = x[0];
        }
    }
}

int pca_blocks(int64_t npix) {
    const int64_t want = (npix + kPcaThreads * 8 - 1) / (kPcaThreads * 8);
    return (int)(want < 1 ? 1 : (want > 608 ? 608 : want));
}

PcaBasis to_basis(int bands, int npc, const double* mean, const double* comps) {
    PcaBasis B{};
    for (int b = 0; b < bands; ++b) B.m[b] = (float)mean[b];
    for (int k = 0; k < npc; ++k)
        for (int b = 0; b < bands; ++b) B.v[k][b] = (float)comps[k * bands + b];
    return B;
}

}  // namespace

// Eigen-decomposition of a symmetric n x n matrix (row-major, n <= 16) by
// cyclic Jacobi rotations (Golub and Van Loan, the classical Jacobi method):
// rows of vecs = eigenvectors, in order of decreasing eigenvalue (ties:
// lower index first), each signed so that its first entry of largest
// magnitude is positive.
void pca_eigen(int n, const double* a_in, double* vals, double* vecs) {
    std::vector<double> a(a_in, a_in + n * n), v(n * n, 0.0);
    for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a[i * n + j] * a[i * n + j];
                if (i != j) off += a[i * n + j] * a[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[p * n + q];
                if (apq == 0.0) continue;
                const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // V <- V J
                    const double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = c * vkp - s * vkq;
                    v[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return a[x * n + x] > a[y * n + y]; });
    for (int r = 0; r < n; ++r) {
        const int col = order[r];
        vals[r] = a[col * n + col];
        int jmax = 0;
        for (int k = 1; k < n; ++k)
            if (std::fabs(v[k * n + col]) > std::fabs(v[jmax * n + col])) jmax = k;
        const double sg = v[jmax * n + col] < 0 ? -1.0 : 1.0;
        for (int k = 0; k < n; ++k) vecs[r * n + k] = sg * v[k * n + col];
    }
}

int pca_fit_blocks(int64_t npix) { return pca_blocks(npix); }

cudaError_t launch_pca_sums(const void* src, xv_dtype dt, int bands, int64_t npix, double* part, int nblk,
                            cudaStream_t st) {
    if (dt == XV_F32) k_pca_sums<float><<<nblk, kPcaThreads, 0, st>>>(static_cast<const float*>(src), bands, npix, part);
    else k_pca_sums<uint16_t><<<nblk, kPcaThreads, 0, st>>>(static_cast<const uint16_t*>(src), bands, npix, part);
    return cudaGetLastError();
}

cudaError_t launch_pca_cov(const void* src, xv_dtype dt, int bands, int64_t npix, const double* mean, double* part,
                           int nblk, cudaStream_t st) {
    PcaMean m{};
    for (int b = 0; b < bands; ++b) m.m[b] = mean[b];
    if (dt == XV_F32) k_pca_cov<float><<<nblk, kPcaThreads, 0, st>>>(static_cast<const float*>(src), bands, npix, m, part);
    else k_pca_cov<uint16_t><<<nblk, kPcaThreads, 0, st>>>(static_cast<const uint16_t*>(src), bands, npix, m, part);
    return cudaGetLastError();
}

cudaError_t launch_pca_project(const void* src, xv_dtype dt, int bands, int npc, int64_t npix, const double* mean,
                               const double* comps, float* dst, cudaStream_t st) {
    const PcaBasis B = to_basis(bands, npc, mean, comps);
    const int nblk = pca_blocks(npix);
    const uintptr_t a = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
    const bool vec = npix % 4 == 0 && a % 16 == 0;
    if (dt == XV_F32) {
        const float* s = static_cast<const float*>(src);
        if (vec) k_pca_project<float, 4><<<nblk, kPcaThreads, 0, st>>>(s, bands, npc, npix, B, dst);
        else k_pca_project<float, 1><<<nblk, kPcaThreads, 0, st>>>(s, bands, npc, npix, B, dst);
    } else {
        const uint16_t* s = static_cast<const uint16_t*>(src);
        if (vec) k_pca_project<uint16_t, 4><<<nblk, kPcaThreads, 0, st>>>(s, bands, npc, npix, B, dst);
        else k_pca_project<uint16_t, 1><<<nblk, kPcaThreads, 0, st>>>(s, bands, npc, npix, B, dst);
    }
    return cudaGetLastError();
}

cudaError_t launch_pca_inverse(const float* z, int npc, int bands, int64_t npix, const double* mean, const double* comps,
                               float* dst, cudaStream_t st) {
    const PcaBasis B = to_basis(bands, npc, mean, comps);
    const uintptr_t a = reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(dst);
    if (npix % 4 == 0 && a % 16 == 0) k_pca_inverse<4><<<pca_blocks(npix), kPcaThreads, 0, st>>>(z, npc, bands, npix, B, dst);
    else k_pca_inverse<1><<<pca_blocks(npix), kPcaThreads, 0, st>>>(z, npc, bands, npix, B, dst);
    return cudaGetLastError();
}

}  // namespace xvh
