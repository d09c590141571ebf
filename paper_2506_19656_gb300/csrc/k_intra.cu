// k_intra.cu -- frame-0 intra coding (the XV_INTRA option): one thread block
// per CU, the CUs of a frame in a wavefront of launches.
//
// Definitions: xv_intra_frame in include/xv.h.  A CU is predicted from its
// reconstructed neighbours (left, top-left, top, top-right; never the
// below-left, which is coded later in raster order), so CU (r, c) waits for
// (r, c-1) and (r-1, c+1): launch w holds the CUs with c + 2 r = w, whose
// neighbours all lie on earlier waves.  In a block: the current samples and
// the 4N + 1 reference samples of each channel (unavailable ones substituted
// as H.265 does), the channel-0 SATD of all 35 modes (one 8 x 8 Hadamard per
// thread and task), the best mode's prediction of all three channels, then
// the transform/quantise/reconstruct of an inter CU on that prediction.
#include <cuda_runtime.h>

#include <cstdint>

#include "dec.cuh"
#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kNT = 256;
constexpr int kModes = 35;
constexpr int kModeBits = 6;  // rate proxy of the mode of an intra CU

// H.265's prediction angle per mode (2..34; 0 planar and 1 DC have none)
__constant__ int c_angle[kModes] = {0,   0,  32, 26, 21, 17, 13, 9,  5,  2,   0,   -2,  -5,  -9, -13, -17, -21, -26,
                                    -32, -26, -21, -17, -13, -9, -5, -2, 0,  2,  5,   9,   13, 17, 21,  26,  32};

// 8192 / angle rounded to the nearest integer, for the negative angles
__device__ __forceinline__ int inv_angle(int a) {
    switch (a) {
        case -2: return -4096;
        case -5: return -1638;
        case -9: return -910;
        case -13: return -630;
        case -17: return -482;
        case -21: return -390;
        case -26: return -315;
        case -32: return -256;
    }
    return 0;
}

// Shared memory after the transform's region: the reference samples of the
// three channels in scan order (sv[i]: i < 2N the left column from the
// bottom up, 2N the corner, then the top row left to right), their
// availability, the DC values, the modes' SATD and the chosen mode.
__host__ __device__ constexpr int intra_nref(int N) { return 4 * N + 1; }
__host__ __device__ constexpr size_t intra_off_ref(int N) { return xvd::align16(xvd::tqr_smem_bytes(N)); }
__host__ __device__ constexpr size_t intra_off_av(int N) { return intra_off_ref(N) + xvd::align16((size_t)3 * intra_nref(N) * 4); }
__host__ __device__ constexpr size_t intra_off_misc(int N) { return intra_off_av(N) + xvd::align16((size_t)3 * intra_nref(N)); }
__host__ __device__ constexpr size_t intra_smem_bytes(int N) { return intra_off_misc(N) + (3 + kModes + 1) * 4; }

// Prediction of sample (x, y) of an N x N block in `mode` from the scan-order
// references sv (dc: the block's DC value).
__device__ __forceinline__ int intra_sample(const int* __restrict__ sv, int N, int L, int mode, int dc, int x, int y) {
    auto left = [&](int j) { return sv[2 * N - 1 - j]; };
    auto top = [&](int j) { return sv[2 * N + 1 + j]; };
    if (mode == 0)
        return ((N - 1 - x) * left(y) + (x + 1) * top(N) + (N - 1 - y) * top(x) + (y + 1) * left(N) + N) >> (L + 1);
    if (mode == 1) return dc;
    const int angle = c_angle[mode];
    const bool vertical = mode >= 18;
    const int pos = vertical ? y : x, along = vertical ? x : y;
    const int idx = ((pos + 1) * angle) >> 5, fact = ((pos + 1) * angle) & 31;
    // main reference k: 0 the corner, k > 0 the side along the direction,
    // k < 0 the other side projected with the inverse angle
    auto refk = [&](int k) {
        if (k == 0) return sv[2 * N];
        if (k > 0) return vertical ? top(k - 1) : left(k - 1);
        const int j = -1 + ((k * inv_angle(angle) + 128) >> 8);
        return vertical ? left(j) : top(j);
    };
    const int k0 = along + idx + 1;
    const int a = refk(k0);
    return fact ? ((32 - fact) * a + fact * refk(k0 + 1) + 16) >> 5 : a;
}

// The reference samples of the CU (r, c) of all three channels from the
// reconstruction rg, in scan order with their availability (inside the plane
// and in a CU coded earlier in raster order), unavailable ones substituted,
// and each channel's DC value.  Called by all threads; ends with a barrier.
template <int N>
__device__ void intra_refs(const uint16_t* __restrict__ rg, int64_t plane, int Hp, int Wp, int r, int c,
                           int* s_ref, unsigned char* s_av, int* s_dc) {
    constexpr int NR = intra_nref(N), L = N == 8 ? 3 : N == 16 ? 4 : N == 32 ? 5 : 6;
    const int tid = threadIdx.x, x0 = c * N, y0 = r * N;
    for (int i = tid; i < 3 * NR; i += kNT) {
        const int ch = i / NR, k = i - ch * NR;
        int x, y;
        if (k < 2 * N) { x = x0 - 1; y = y0 + 2 * N - 1 - k; }
        else if (k == 2 * N) { x = x0 - 1; y = y0 - 1; }
        else { x = x0 + k - 2 * N - 1; y = y0 - 1; }
        const bool in = x >= 0 && y >= 0 && x < Wp && y < Hp;
        const bool coded = in && (y / N < r || (y / N == r && x / N < c));
        s_av[i] = coded;
        s_ref[i] = coded ? rg[ch * plane + (int64_t)y * Wp + x] : 0;
    }
    __syncthreads();
    // substitution along the scan, one thread per channel
    if (tid < 3) {
        int* sv = s_ref + tid * NR;
        const unsigned char* av = s_av + tid * NR;
        int first = -1;
        for (int k = 0; k < NR && first < 0; ++k)
            if (av[k]) first = k;
        if (first < 0) {
            for (int k = 0; k < NR; ++k) sv[k] = xvd::kFlat;
        } else {
            if (!av[0]) sv[0] = sv[first];
            for (int k = 1; k < NR; ++k)
                if (!av[k]) sv[k] = sv[k - 1];
        }
    }
    __syncthreads();
    // DC per channel: (sum of the N left and N top samples + N) >> (log2 N + 1)
    if (tid < 96) {
        const int ch = tid >> 5, lane = tid & 31;
        const int* sv = s_ref + ch * NR;
        int s = 0;
        for (int j = lane; j < N; j += 32) s += sv[2 * N - 1 - j] + sv[2 * N + 1 + j];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) s_dc[ch] = (s + N) >> (L + 1);
    }
    __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kNT)
k_intra_cu(const uint16_t* __restrict__ cur, int64_t gstride, int Hp, int Wp, int wave, int r_lo, int qp,
           unsigned tu_mask, int64_t lf8, int16_t* mv, int64_t pu_gstride, uint16_t* recon, int16_t* levels,
           uint8_t* tu_log2, uint64_t* bits, int64_t bits_gstride) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NN = N * N, NR = intra_nref(N), L = N == 8 ? 3 : N == 16 ? 4 : N == 32 ? 5 : 6;
    const int tid = threadIdx.x, g = blockIdx.y;
    const int r = r_lo + blockIdx.x, c = wave - 2 * r;
    const int x0 = c * N, y0 = r * N, nx = Wp / N;
    const int64_t plane = (int64_t)Hp * Wp;
    const uint16_t* cg = cur + g * gstride;
    uint16_t* rg = recon + g * gstride;
    uint16_t* s_cur = reinterpret_cast<uint16_t*>(smem);
    uint16_t* s_pred = s_cur + 3 * NN;
    int* s_ref = reinterpret_cast<int*>(smem + intra_off_ref(N));
    unsigned char* s_av = smem + intra_off_av(N);
    int* s_dc = reinterpret_cast<int*>(smem + intra_off_misc(N));
    unsigned* s_satd = reinterpret_cast<unsigned*>(s_dc + 3);
    int* s_best = reinterpret_cast<int*>(s_satd + kModes);

    // current samples; reference samples with their availability (inside the
    // plane and in a CU coded earlier in raster order)
    for (int i = tid; i < 3 * NN; i += kNT) {
        const int ch = i / NN, y = (i / N) % N, x = i % N;
        s_cur[i] = cg[ch * plane + (int64_t)(y0 + y) * Wp + x0 + x];
    }
    if (tid < kModes) s_satd[tid] = 0u;  // ordered by intra_refs' barriers
    intra_refs<N>(rg, plane, Hp, Wp, r, c, s_ref, s_av, s_dc);
    // channel-0 SATD of every mode: one 8 x 8 block of one mode per task
    {
        constexpr int NB = (N / 8) * (N / 8);
        for (int t = tid; t < kModes * NB; t += kNT) {
            const int m = t / NB, b = t - m * NB;
            const int bx = (b % (N / 8)) * 8, by = (b / (N / 8)) * 8;
            int d[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    d[i][j] = (int)s_cur[(by + i) * N + bx + j] - intra_sample(s_ref, N, L, m, s_dc[0], bx + j, by + i);
#pragma unroll
            for (int i = 0; i < 8; ++i) xvd::hadamard8_row(d[i]);
            unsigned sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int col[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) col[i] = d[i][j];
                xvd::hadamard8_row(col);
#pragma unroll
                for (int i = 0; i < 8; ++i) sum += (unsigned)abs(col[i]);
            }
            atomicAdd(&s_satd[m], (sum + 2) >> 2);
        }
    }
    __syncthreads();
    if (tid == 0) {  // the least SATD, the lower mode on ties
        int best = 0;
        for (int m = 1; m < kModes; ++m)
            if (s_satd[m] < s_satd[best]) best = m;
        *s_best = best;
    }
    __syncthreads();
    const int mode = *s_best;
    for (int i = tid; i < 3 * NN; i += kNT) {
        const int ch = i / NN, y = (i / N) % N, x = i % N;
        s_pred[i] = (uint16_t)intra_sample(s_ref + ch * NR, N, L, mode, s_dc[ch], x, y);
    }
    __syncthreads();
    const int cu = r * nx + c;
    const int64_t o = g * pu_gstride + cu;
    const uint32_t b = xvd::tqr_cu<N, kNT, false, true>(nullptr, nullptr, plane, Hp, Wp, x0, y0, 0, 0, qp, tu_mask,
                                                        lf8, rg, levels ? levels + g * gstride : nullptr,
                                                        tu_log2 ? tu_log2 + o : nullptr, smem);
    if (tid == 0) {
        mv[2 * o] = (int16_t)mode;
        mv[2 * o + 1] = 0;
        atomicAdd(reinterpret_cast<unsigned long long*>(bits + g * bits_gstride),
                  (unsigned long long)(b + kModeBits));
    }
}

// Decoding of frame 0 with intra prediction: the CU's levels, its references
// from the decoded neighbours, the prediction with the stored mode
// (mode_mv[cu][0], clamped to 0..34), then dec_cu on that prediction.
__host__ __device__ constexpr size_t intra_dec_off_ref(int N) { return xvd::align16(xvd::dec_smem_bytes(N)); }
__host__ __device__ constexpr size_t intra_dec_smem_bytes(int N) {
    return intra_dec_off_ref(N) + xvd::align16((size_t)3 * intra_nref(N) * 4) + xvd::align16((size_t)3 * intra_nref(N)) +
           4 * 4;
}

template <int N>
__global__ void __launch_bounds__(kNT)
k_intra_dec_cu(const int16_t* __restrict__ levels, int64_t gstride, int Hp, int Wp, int wave, int r_lo, int qp,
               const int16_t* __restrict__ mode_mv, int64_t pu_gstride, const uint8_t* __restrict__ tu_log2,
               uint16_t* recon, uint64_t* bits, int64_t bits_gstride) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NN = N * N, NR = intra_nref(N), L = N == 8 ? 3 : N == 16 ? 4 : N == 32 ? 5 : 6;
    const int tid = threadIdx.x, g = blockIdx.y;
    const int r = r_lo + blockIdx.x, c = wave - 2 * r;
    const int x0 = c * N, y0 = r * N, nx = Wp / N;
    const int64_t plane = (int64_t)Hp * Wp;
    const int16_t* lg = levels + g * gstride;
    uint16_t* rg = recon + g * gstride;
    int16_t* s_lev = reinterpret_cast<int16_t*>(smem);
    uint16_t* s_pred = reinterpret_cast<uint16_t*>(s_lev + 3 * NN);
    int* s_ref = reinterpret_cast<int*>(smem + intra_dec_off_ref(N));
    unsigned char* s_av = reinterpret_cast<unsigned char*>(s_ref + 3 * NR);
    int* s_dc = reinterpret_cast<int*>(smem + intra_dec_off_ref(N) + xvd::align16((size_t)3 * NR * 4) +
                                       xvd::align16((size_t)3 * NR));
    for (int i = tid; i < 3 * NN; i += kNT) {
        const int ch = i / NN, y = (i / N) % N, x = i % N;
        s_lev[i] = lg[ch * plane + (int64_t)(y0 + y) * Wp + x0 + x];
    }
    intra_refs<N>(rg, plane, Hp, Wp, r, c, s_ref, s_av, s_dc);
    const int cu = r * nx + c;
    const int64_t o = g * pu_gstride + cu;
    const int m = mode_mv[2 * o];
    const int mode = m < 0 ? 0 : (m > kModes - 1 ? kModes - 1 : m);
    for (int i = tid; i < 3 * NN; i += kNT) {
        const int ch = i / NN, y = (i / N) % N, x = i % N;
        s_pred[i] = (uint16_t)intra_sample(s_ref + ch * NR, N, L, mode, s_dc[ch], x, y);
    }
    __syncthreads();
    const uint32_t b = xvd::dec_cu<N, kNT, false, true>(nullptr, nullptr, plane, Hp, Wp, x0, y0, 0, 0, tu_log2[o], qp,
                                                        rg, smem);
    if (tid == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(bits + g * bits_gstride), (unsigned long long)(b + kModeBits));
}

// The wave w of a frame of nx x ny CUs: its first CU row and CU count.
inline void wave_rows(int w, int nx, int ny, int& r_lo, int& count) {
    const int a = w - (nx - 1);
    r_lo = a > 0 ? (a + 1) / 2 : 0;
    const int r_hi = w / 2 < ny - 1 ? w / 2 : ny - 1;
    count = r_hi - r_lo + 1;
}

template <int N>
cudaError_t intra_dec_n(const int16_t* levels, int G, int64_t gstride, int Hp, int Wp, int qp, const int16_t* mode_mv,
                        int64_t pu_gstride, const uint8_t* tu_log2, uint16_t* recon, uint64_t* bits,
                        int64_t bits_gstride, cudaStream_t st, uint64_t* launches) {
    const size_t smem = intra_dec_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_intra_dec_cu<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nx = Wp / N, ny = Hp / N;
    for (int w = 0; w < (nx - 1) + 2 * (ny - 1) + 1; ++w) {
        int r_lo, count;
        wave_rows(w, nx, ny, r_lo, count);
        if (count < 1) continue;
        k_intra_dec_cu<N><<<dim3(count, G), kNT, smem, st>>>(levels, gstride, Hp, Wp, w, r_lo, qp, mode_mv, pu_gstride,
                                                             tu_log2, recon, bits, bits_gstride);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

template <int N>
cudaError_t intra_n(const uint16_t* cur, int G, int64_t gstride, int Hp, int Wp, const xv_params* p, int16_t* mv,
                    int64_t pu_gstride, uint16_t* recon, int16_t* levels, uint8_t* tu_log2, uint64_t* bits,
                    int64_t bits_gstride, cudaStream_t st, uint64_t* launches) {
    const size_t smem = intra_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_intra_cu<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nx = Wp / N, ny = Hp / N;
    const int waves = (nx - 1) + 2 * (ny - 1) + 1;
    for (int w = 0; w < waves; ++w) {
        const int a = w - (nx - 1);
        const int r_lo = a > 0 ? (a + 1) / 2 : 0, r_hi = w / 2 < ny - 1 ? w / 2 : ny - 1;
        if (r_hi < r_lo) continue;
        dim3 grid(r_hi - r_lo + 1, G);
        k_intra_cu<N><<<grid, kNT, smem, st>>>(cur, gstride, Hp, Wp, w, r_lo, p->qp, p->tu_mask, p->lambda_fp8, mv,
                                               pu_gstride, recon, levels, tu_log2, bits, bits_gstride);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_intra_frame(const uint16_t* cur, int G, int64_t gstride, int Hp, int Wp, const xv_params* p,
                               int16_t* mv, int64_t pu_gstride, uint16_t* recon, int16_t* levels, uint8_t* tu_log2,
                               uint64_t* bits, int64_t bits_gstride, cudaStream_t st, uint64_t* launches) {
    switch (p->ctu) {
        case 8: return intra_n<8>(cur, G, gstride, Hp, Wp, p, mv, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st, launches);
        case 16: return intra_n<16>(cur, G, gstride, Hp, Wp, p, mv, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st, launches);
        case 32: return intra_n<32>(cur, G, gstride, Hp, Wp, p, mv, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st, launches);
        case 64: return intra_n<64>(cur, G, gstride, Hp, Wp, p, mv, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st, launches);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_intra_decode_frame(const int16_t* levels, int G, int64_t gstride, int Hp, int Wp, int ctu, int qp,
                                      const int16_t* mode_mv, int64_t pu_gstride, const uint8_t* tu_log2,
                                      uint16_t* recon, uint64_t* bits, int64_t bits_gstride, cudaStream_t st,
                                      uint64_t* launches) {
    switch (ctu) {
        case 8: return intra_dec_n<8>(levels, G, gstride, Hp, Wp, qp, mode_mv, pu_gstride, tu_log2, recon, bits, bits_gstride, st, launches);
        case 16: return intra_dec_n<16>(levels, G, gstride, Hp, Wp, qp, mode_mv, pu_gstride, tu_log2, recon, bits, bits_gstride, st, launches);
        case 32: return intra_dec_n<32>(levels, G, gstride, Hp, Wp, qp, mode_mv, pu_gstride, tu_log2, recon, bits, bits_gstride, st, launches);
        case 64: return intra_dec_n<64>(levels, G, gstride, Hp, Wp, qp, mode_mv, pu_gstride, tu_log2, recon, bits, bits_gstride, st, launches);
    }
    return cudaErrorInvalidValue;
}

}  // namespace xvh
