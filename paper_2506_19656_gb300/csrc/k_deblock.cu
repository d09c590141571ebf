// k_deblock.cu -- in-loop deblocking of reconstructed frames (the XV_DEBLOCK
// option): the H.265 luma deblocking filter applied alike to all three
// channels.
//
// Definitions: xv_deblock_frame in include/xv.h.  Edges lie on the 8 x 8 grid
// where a CU or a TU of the CU containing the edge's q side begins.  Per
// 4-sample segment the boundary strength is 2 for intra CUs, 1 when the TU on
// either side has a non-zero level in any channel (k_cbf marks those per 4 x 4
// block) or the two CUs' vectors differ by 4 quarter samples or more, else 0.
// Every vertical edge of the frame is filtered first (k_deblock<true>; edges 8
// apart touch at most 3 samples each side, so segments never overlap), then
// every horizontal edge on that result (k_deblock<false>).  One thread per
// segment filters it in all three channels.
#include <cuda_runtime.h>

#include <cstdint>

#include "xv_internal.h"

namespace xvh {
namespace {

// beta' (QP 0..51) and tC' (QP 0..53) of H.265, for 8-bit samples
__constant__ int c_beta[52] = {0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  6,  7,
                               8,  9,  10, 11, 12, 13, 14, 15, 16, 17, 18, 20, 22, 24, 26, 28, 30, 32,
                               34, 36, 38, 40, 42, 44, 46, 48, 50, 52, 54, 56, 58, 60, 62, 64};
__constant__ int c_tc[54] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,  1,  1,  1,  1,  1,  1,  1,  1, 1,
                             2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 5, 5, 6, 6, 7, 8, 9, 10, 11, 13, 14, 16, 18, 20, 22, 24};
constexpr int kBitShift = 2;  // 10-bit samples: beta and tC scaled by 2^(10 - 8)
constexpr int kMax = 1023;

__device__ __forceinline__ int clip3(int lo, int hi, int v) { return v < lo ? lo : (v > hi ? hi : v); }

// TU size from a stored log2 value, kept inside 4..ctu whatever the caller's
// data hold (every index below relies on it)
__device__ __forceinline__ int tu_size(uint8_t l, int ctu) {
    const int ts = 1 << (l < 2 ? 2 : (l > 6 ? 6 : l));
    return ts > ctu ? ctu : ts;
}

// Coded-block map: cbf[(y / 4) * (Wp / 4) + x / 4] = 1 when the TU holding
// sample (x, y) has a non-zero level in any channel.  One block per CU.
__global__ void k_cbf(const int16_t* __restrict__ levels, int64_t gstride, int Hp, int Wp, int ctu,
                      const uint8_t* __restrict__ tu_log2, int64_t pu_gstride, uint8_t* cbf, int64_t cbf_gstride) {
    __shared__ int s_flag[256];  // TUs of a CU: at most (64 / 4)^2
    const int cu = blockIdx.x, g = blockIdx.y, nx = Wp / ctu;
    const int x0 = (cu % nx) * ctu, y0 = (cu / nx) * ctu;
    const int TS = tu_size(tu_log2[g * pu_gstride + cu], ctu), side = ctu / TS;
    const int64_t plane = (int64_t)Hp * Wp;
    const int16_t* lg = levels + g * gstride;
    for (int i = threadIdx.x; i < side * side; i += blockDim.x) s_flag[i] = 0;
    __syncthreads();
    const int nn = ctu * ctu;
    for (int i = threadIdx.x; i < 3 * nn; i += blockDim.x) {
        const int ch = i / nn, y = (i / ctu) % ctu, x = i % ctu;
        if (lg[ch * plane + (int64_t)(y0 + y) * Wp + x0 + x] != 0) s_flag[(y / TS) * side + x / TS] = 1;
    }
    __syncthreads();
    const int q = ctu / 4;
    for (int i = threadIdx.x; i < q * q; i += blockDim.x) {
        const int bx = i % q, by = i / q;
        cbf[g * cbf_gstride + (int64_t)(y0 / 4 + by) * (Wp / 4) + x0 / 4 + bx] =
            (uint8_t)s_flag[((by * 4) / TS) * side + (bx * 4) / TS];
    }
}

// One 4-sample segment of one channel: v[k][i], line k, i = 0..3 the p side
// (p3 p2 p1 p0), 4..7 the q side (q0 q1 q2 q3); filtered in place.
__device__ void filter_segment(int (&v)[4][8], int beta, int tc) {
    auto p = [&](int k, int i) -> int& { return v[k][3 - i]; };
    auto q = [&](int k, int i) -> int& { return v[k][4 + i]; };
    const int dp0 = abs(p(0, 2) - 2 * p(0, 1) + p(0, 0)), dp3 = abs(p(3, 2) - 2 * p(3, 1) + p(3, 0));
    const int dq0 = abs(q(0, 2) - 2 * q(0, 1) + q(0, 0)), dq3 = abs(q(3, 2) - 2 * q(3, 1) + q(3, 0));
    if (dp0 + dq0 + dp3 + dq3 >= beta) return;
    auto strong_line = [&](int k, int dpq) {
        return 2 * dpq < (beta >> 2) && abs(p(k, 3) - p(k, 0)) + abs(q(k, 0) - q(k, 3)) < (beta >> 3) &&
               abs(p(k, 0) - q(k, 0)) < ((5 * tc + 1) >> 1);
    };
    const bool strong = strong_line(0, dp0 + dq0) && strong_line(3, dp3 + dq3);
    const bool dEp = dp0 + dp3 < ((beta + (beta >> 1)) >> 3), dEq = dq0 + dq3 < ((beta + (beta >> 1)) >> 3);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p0 = p(k, 0), p1 = p(k, 1), p2 = p(k, 2), p3 = p(k, 3);
        const int q0 = q(k, 0), q1 = q(k, 1), q2 = q(k, 2), q3 = q(k, 3);
        if (strong) {
            const int t2 = 2 * tc;
            p(k, 0) = clip3(p0 - t2, p0 + t2, (p2 + 2 * p1 + 2 * p0 + 2 * q0 + q1 + 4) >> 3);
            p(k, 1) = clip3(p1 - t2, p1 + t2, (p2 + p1 + p0 + q0 + 2) >> 2);
            p(k, 2) = clip3(p2 - t2, p2 + t2, (2 * p3 + 3 * p2 + p1 + p0 + q0 + 4) >> 3);
            q(k, 0) = clip3(q0 - t2, q0 + t2, (p1 + 2 * p0 + 2 * q0 + 2 * q1 + q2 + 4) >> 3);
            q(k, 1) = clip3(q1 - t2, q1 + t2, (p0 + q0 + q1 + q2 + 2) >> 2);
            q(k, 2) = clip3(q2 - t2, q2 + t2, (p0 + q0 + q1 + 3 * q2 + 2 * q3 + 4) >> 3);
        } else {
            int delta = (9 * (q0 - p0) - 3 * (q1 - p1) + 8) >> 4;
            if (abs(delta) >= 10 * tc) continue;
            delta = clip3(-tc, tc, delta);
            p(k, 0) = clip3(0, kMax, p0 + delta);
            q(k, 0) = clip3(0, kMax, q0 - delta);
            const int h = tc >> 1;
            if (dEp) p(k, 1) = clip3(0, kMax, p1 + clip3(-h, h, (((p2 + p0 + 1) >> 1) - p1 + delta) >> 1));
            if (dEq) q(k, 1) = clip3(0, kMax, q1 + clip3(-h, h, (((q2 + q0 + 1) >> 1) - q1 - delta) >> 1));
        }
    }
}

// kVertical: the segments of the vertical edges x = 8, 16, ... (4 rows each);
// else of the horizontal edges y = 8, 16, ... (4 columns each).
template <bool kVertical>
__global__ void k_deblock(uint16_t* rec, int64_t gstride, int G, int Hp, int Wp, int ctu, int qp,
                          const uint8_t* __restrict__ tu_log2, int64_t pu_gstride, const uint8_t* __restrict__ cbf,
                          int64_t cbf_gstride, const int16_t* __restrict__ mv, int intra) {
    const int E = kVertical ? Wp : Hp, O = kVertical ? Hp : Wp;
    const int nedge = E / 8 - 1, nseg = O / 4, nx = Wp / ctu;
    const int64_t total = (int64_t)G * nedge * nseg, plane = (int64_t)Hp * Wp;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(it / ((int64_t)nedge * nseg));
        const int rem = (int)(it - (int64_t)g * nedge * nseg);
        // consecutive threads take neighbouring segments along the rows: the
        // edges of one row band for vertical edges, the 4-column segments of
        // one edge for horizontal ones (their sample windows are contiguous)
        const int e = kVertical ? 8 * (rem % nedge + 1) : 8 * (rem / nseg + 1);
        const int o = kVertical ? 4 * (rem / nedge) : 4 * (rem % nseg);
        // the q-side sample and the p-side sample of the segment's first line
        const int xq = kVertical ? e : o, yq = kVertical ? o : e;
        const int xp = kVertical ? e - 1 : o, yp = kVertical ? o : e - 1;
        const int cuq = (yq / ctu) * nx + xq / ctu, cup = (yp / ctu) * nx + xp / ctu;
        const uint8_t* tug = tu_log2 + g * pu_gstride;
        if (e % ctu != 0 && e % tu_size(tug[cuq], ctu) != 0) continue;  // not a CU or TU boundary
        int bs = 0;
        if (intra) {
            bs = 2;
        } else {
            const uint8_t* cg = cbf + g * cbf_gstride;
            if (cg[(int64_t)(yq / 4) * (Wp / 4) + xq / 4] || cg[(int64_t)(yp / 4) * (Wp / 4) + xp / 4]) {
                bs = 1;
            } else if (cup != cuq) {
                const int16_t* mg = mv + 2 * g * pu_gstride;
                if (abs(mg[2 * cup] - mg[2 * cuq]) >= 4 || abs(mg[2 * cup + 1] - mg[2 * cuq + 1]) >= 4) bs = 1;
            }
        }
        if (bs == 0) continue;
        const int beta = c_beta[clip3(0, 51, qp)] << kBitShift;
        const int tc = c_tc[clip3(0, 53, qp + 2 * (bs - 1))] << kBitShift;
        uint16_t* rg = rec + g * gstride;
        for (int ch = 0; ch < 3; ++ch) {
            uint16_t* pl = rg + ch * plane;
            int v[4][8];
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    v[k][i] = kVertical ? pl[(int64_t)(o + k) * Wp + e - 4 + i] : pl[(int64_t)(e - 4 + i) * Wp + o + k];
            int w[4][8];
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int i = 0; i < 8; ++i) w[k][i] = v[k][i];
            filter_segment(w, beta, tc);
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int i = 1; i < 7; ++i)  // p3 and q3 never change
                    if (w[k][i] != v[k][i]) {
                        if (kVertical) pl[(int64_t)(o + k) * Wp + e - 4 + i] = (uint16_t)w[k][i];
                        else pl[(int64_t)(e - 4 + i) * Wp + o + k] = (uint16_t)w[k][i];
                    }
        }
    }
}

int grid_for(int64_t items) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (items + 255) / 256, cap = (int64_t)sms * 16;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_deblock_frame(uint16_t* recon, int G, int64_t gstride, int Hp, int Wp, int ctu, int qp,
                                 const uint8_t* tu_log2, int64_t pu_gstride, const int16_t* levels,
                                 const int16_t* mv, int intra, uint8_t* cbf, cudaStream_t st, uint64_t* launches) {
    const int64_t cbf_gstride = (int64_t)(Hp / 4) * (Wp / 4);
    if (!intra) {
        k_cbf<<<dim3((Hp / ctu) * (Wp / ctu), G), 128, 0, st>>>(levels, gstride, Hp, Wp, ctu, tu_log2, pu_gstride,
                                                                cbf, cbf_gstride);
        if (launches) ++*launches;
    }
    const int64_t nv = (int64_t)G * (Wp / 8 - 1) * (Hp / 4), nh = (int64_t)G * (Hp / 8 - 1) * (Wp / 4);
    if (nv > 0) {
        k_deblock<true><<<grid_for(nv), 256, 0, st>>>(recon, gstride, G, Hp, Wp, ctu, qp, tu_log2, pu_gstride, cbf,
                                                      cbf_gstride, mv, intra);
        if (launches) ++*launches;
    }
    if (nh > 0) {
        k_deblock<false><<<grid_for(nh), 256, 0, st>>>(recon, gstride, G, Hp, Wp, ctu, qp, tu_log2, pu_gstride, cbf,
                                                       cbf_gstride, mv, intra);
        if (launches) ++*launches;
    }
    return cudaGetLastError();
}

}  // namespace xvh
