// me.cuh -- motion estimation of one PU by one thread block (device code).
//
// Integer full search over [-R, R]^2 on channel 0 with SAD + motion cost,
// then quarter-sample refinement with Hadamard SATD + motion cost; the
// definitions are those of xv_motion_search in include/xv.h.
//
// Layout in shared memory:
//   win  int32 [WW][S]  reference window, WW = N + 2R + 8 rows/columns around
//                       the PU (margin R + 4: the 8-tap filter at vectors up
//                       to +-(R + 3/4)), coordinates clamped to the plane when
//                       loaded -- so the search itself never branches on
//                       borders.  S >= WW with S = 4 (mod 8): rows of
//                       consecutive lanes fall in distinct 16-byte bank
//                       groups for 128-bit loads.
//   blk  int32 [N][N]   the PU's channel-0 samples.
//   hp   int16 [3][N+8][N]  horizontally filtered columns for the three
//                       x-vectors of one refinement stage.
// Work split of the integer search: a unit is one candidate row dy and 8
// consecutive dx; consecutive lanes take consecutive dy (distinct window
// rows), so the reference loads are conflict-free and the current-block loads
// are warp-wide broadcasts.  Each lane keeps its best 64-bit key
// (J << 32 | raster index); a block-wide min gives the winner and the
// tie-break of the definition.
#pragma once
#include <cstdint>
#include "xv_dev.cuh"

namespace xvd {

struct MeResult {
    int mvx_int, mvy_int;  // integer vector (pixels)
    uint32_t cost_int;
    int mvx, mvy;          // final vector (quarter samples)
    uint32_t cost;
};

__host__ __device__ constexpr int me_win(int N, int R) { return N + 2 * R + 8; }
__host__ __device__ constexpr int me_stride(int N, int R) {
    return ((me_win(N, R) + 3) / 8) * 8 + 4;  // smallest S >= WW with S % 8 == 4
}
// Byte offsets of the shared-memory regions (every region 16-byte aligned).
__host__ __device__ constexpr size_t me_align16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ constexpr size_t me_off_blk(int N, int R) { return me_align16((size_t)me_win(N, R) * me_stride(N, R) * 4); }
__host__ __device__ constexpr size_t me_off_hp(int N, int R) { return me_off_blk(N, R) + me_align16((size_t)N * N * 4); }
__host__ __device__ constexpr size_t me_off_red(int N, int R) { return me_off_hp(N, R) + me_align16((size_t)3 * (N + 8) * N * 2); }
__host__ __device__ constexpr size_t me_off_satd(int N, int R) { return me_off_red(N, R) + 64 * 8; }
__host__ __device__ constexpr size_t me_smem_bytes(int N, int R) { return me_off_satd(N, R) + 16 * 4; }

template <int NT>
__device__ __forceinline__ uint64_t block_min_u64(uint64_t v, uint64_t* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < NT / 32 ? red[lane] : ~0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w < v ? w : v;
        }
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

// SAD of 8 horizontally adjacent candidates over one block row, 16 columns at
// a time: cur[c] against ref[c + k], k = 0..7.
template <int W>
__device__ __forceinline__ void row_sad8(const int* __restrict__ crow, const int* __restrict__ rrow,
                                         uint32_t (&sad)[8]) {
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += 16) {
        constexpr int CW = W < 16 ? W : 16;
        int cv[CW], rv[CW + 8];
#pragma unroll
        for (int i = 0; i < CW; i += 4) {
            int4 t = *reinterpret_cast<const int4*>(crow + c0 + i);
            cv[i] = t.x; cv[i + 1] = t.y; cv[i + 2] = t.z; cv[i + 3] = t.w;
        }
#pragma unroll
        for (int i = 0; i < CW + 8; i += 4) {
            int4 t = *reinterpret_cast<const int4*>(rrow + c0 + i);
            rv[i] = t.x; rv[i + 1] = t.y; rv[i + 2] = t.z; rv[i + 3] = t.w;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < CW; ++c) sad[k] = __sad(cv[c], rv[c + k], sad[k]);
    }
}

// In-register 8-point Hadamard (Sylvester order) of v.
__device__ __forceinline__ void hadamard8_row(int (&v)[8]) {
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!(i & h)) {
                int a = v[i], b = v[i + h];
                v[i] = a + b;
                v[i + h] = a - b;
            }
}

// Refinement stage: evaluate `ncand` quarter-sample candidates around
// (cx, cy) with step s (their vectors in cand_x/cand_y, all within one
// column-set of three x-vectors cx - s, cx, cx + s), SATD summed into satd[].
template <int N, int NT>
__device__ void satd_stage(const int* __restrict__ win, int S, int R, const int* __restrict__ blk,
                           int16_t* __restrict__ hp, int cx, int cy, int s, const int* cand_x,
                           const int* cand_y, int ncand, uint32_t* satd) {
    const int tid = threadIdx.x;
    const int iy_min = (cy - s) >> 2, iy_max = (cy + s) >> 2;
    const int rbase = iy_min - 3;          // block-relative row of hp row 0
    const int nr = N + 7 + (iy_max - iy_min);
    // 1. horizontal pass for the three x-vectors (raw samples for phase 0)
    for (int idx = tid; idx < 3 * nr * N; idx += NT) {
        int j = idx / (nr * N), rem = idx - j * nr * N;
        int r = rem / N, x = rem - r * N;
        int m = cx + (j - 1) * s;
        int hx = m & 3, ix = m >> 2;
        const int* wr = win + (rbase + r + R + 4) * S + (x + ix + R + 4);
        int v;
        if (hx == 0) {
            v = wr[0];
        } else {
            int acc = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) acc += luma_tap(hx, i) * wr[i - 3];
            v = acc >> kShift1;
        }
        hp[(j * (N + 8) + r) * N + x] = (int16_t)v;
    }
    for (int k = tid; k < ncand; k += NT) satd[k] = 0;
    __syncthreads();
    // 2. one 8x8 sub-block of one candidate per 8 lanes (lane = row)
    constexpr int NB = (N / 8) * (N / 8);
    const int lane8 = tid & 7;
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    for (int task = tid >> 3; task < ncand * NB; task += NT / 8) {
        int k = task / NB, b = task - k * NB;
        int by = (b / (N / 8)) * 8, bx = (b % (N / 8)) * 8;
        int mvx = cand_x[k], mvy = cand_y[k];
        int j = (mvx - cx) / s + 1;
        int hx = mvx & 3, fy = mvy & 3, iy = mvy >> 2;
        int y = by + lane8;
        const int16_t* col = hp + (size_t)j * (N + 8) * N + bx;
        int r0 = y + iy - 3 - rbase;  // hp row of tap 0
        int d[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            int v;
            if (fy == 0) {
                int a = col[(r0 + 3) * N + x];
                v = hx == 0 ? a << kShift3 : a;
            } else {
                int acc = 0;
#pragma unroll
                for (int t = 0; t < 8; ++t) acc += luma_tap(fy, t) * (int)col[(r0 + t) * N + x];
                v = hx == 0 ? acc >> kShift1 : acc >> kShift2;
            }
            d[x] = blk[y * N + bx + x] - wp_round(v);
        }
        hadamard8_row(d);
        // vertical transform across the 8 lanes of the group
#pragma unroll
        for (int h = 1; h < 8; h <<= 1) {
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                int o = __shfl_xor_sync(gmask, d[x], h);
                d[x] = (lane8 & h) ? o - d[x] : d[x] + o;
            }
        }
        int sum = 0;
#pragma unroll
        for (int x = 0; x < 8; ++x) sum += d[x] < 0 ? -d[x] : d[x];
        sum += __shfl_xor_sync(gmask, sum, 1);
        sum += __shfl_xor_sync(gmask, sum, 2);
        sum += __shfl_xor_sync(gmask, sum, 4);
        if (lane8 == 0) atomicAdd(&satd[k], (uint32_t)((sum + 2) >> 2));
    }
    __syncthreads();
}

// Motion estimation of the PU at (x0, y0).  cur0/ref0: channel-0 planes.
// Must be called by all NT threads of the block; smem holds me_smem_bytes.
template <int N, int NT, bool kCoherent = false>
__device__ MeResult me_pu(const uint16_t* __restrict__ cur0, const uint16_t* __restrict__ ref0,
                          int Hp, int Wp, int x0, int y0, int R, int64_t lmv, unsigned char* smem) {
    static_assert(N % 8 == 0, "PU size must be a multiple of 8");
    const int tid = threadIdx.x;
    const int WW = me_win(N, R), S = me_stride(N, R);
    int* win = reinterpret_cast<int*>(smem);
    int* blk = reinterpret_cast<int*>(smem + me_off_blk(N, R));
    int16_t* hp = reinterpret_cast<int16_t*>(smem + me_off_hp(N, R));
    uint64_t* red = reinterpret_cast<uint64_t*>(smem + me_off_red(N, R));
    uint32_t* satd = reinterpret_cast<uint32_t*>(smem + me_off_satd(N, R));

    // window with clamped coordinates, and the current block
    const int wx0 = x0 - R - 4, wy0 = y0 - R - 4;
    for (int idx = tid; idx < WW * WW; idx += NT) {
        int r = idx / WW, c = idx - r * WW;
        int yy = min(max(wy0 + r, 0), Hp - 1), xx = min(max(wx0 + c, 0), Wp - 1);
        win[r * S + c] = ld_ref<kCoherent>(ref0 + (size_t)yy * Wp + xx);
    }
    for (int idx = tid; idx < N * N; idx += NT) {
        int r = idx / N, c = idx - r * N;
        blk[idx] = __ldg(cur0 + (size_t)(y0 + r) * Wp + x0 + c);
    }
    __syncthreads();

    // ---- integer full search
    const int side = 2 * R + 1;
    const int ngx = (side + 7) / 8;
    uint64_t best = ~0ull;
    for (int u = tid; u < side * ngx; u += NT) {
        int gx = u / side;
        int dy = u - gx * side - R;
        int dx0 = gx * 8 - R;
        uint32_t sad[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int* wrow = win + (dy + R + 4) * S + (dx0 + R + 4);
#pragma unroll 2
        for (int r = 0; r < N; ++r) row_sad8<N>(blk + r * N, wrow + r * S, sad);
        const uint32_t rowbase = (uint32_t)((dy + R) * side);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int dx = dx0 + k;
            if (dx <= R) {
                uint64_t J = (uint64_t)sad[k] + mv_cost(4 * dx, 4 * dy, lmv);
                uint64_t key = (J << 32) | (rowbase + (uint32_t)(dx + R));
                best = key < best ? key : best;
            }
        }
    }
    best = block_min_u64<NT>(best, red);
    MeResult res;
    {
        int idx = (int)(best & 0xffffffffu);
        res.mvy_int = idx / side - R;
        res.mvx_int = idx - (idx / side) * side - R;
        res.cost_int = (uint32_t)(best >> 32);
    }

    // ---- quarter-sample refinement: centre + 8 half-sample, then 8 quarter
    const int ring_x[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    const int ring_y[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    int cx = 4 * res.mvx_int, cy = 4 * res.mvy_int;
    int cand_x[9], cand_y[9];
    cand_x[0] = cx; cand_y[0] = cy;
#pragma unroll
    for (int k = 0; k < 8; ++k) { cand_x[k + 1] = cx + 2 * ring_x[k]; cand_y[k + 1] = cy + 2 * ring_y[k]; }
    satd_stage<N, NT>(win, S, R, blk, hp, cx, cy, 2, cand_x, cand_y, 9, satd);
    uint32_t bJ = satd[0] + mv_cost(cx, cy, lmv);
    int bx = cx, by = cy;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        uint32_t J = satd[k] + mv_cost(cand_x[k], cand_y[k], lmv);
        if (J < bJ) { bJ = J; bx = cand_x[k]; by = cand_y[k]; }
    }
    __syncthreads();
    cx = bx; cy = by;
#pragma unroll
    for (int k = 0; k < 8; ++k) { cand_x[k] = cx + ring_x[k]; cand_y[k] = cy + ring_y[k]; }
    satd_stage<N, NT>(win, S, R, blk, hp, cx, cy, 1, cand_x, cand_y, 8, satd);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t J = satd[k] + mv_cost(cand_x[k], cand_y[k], lmv);
        if (J < bJ) { bJ = J; bx = cand_x[k]; by = cand_y[k]; }
    }
    __syncthreads();
    res.mvx = bx;
    res.mvy = by;
    res.cost = bJ;
    return res;
}

}  // namespace xvd
