// me.cuh -- motion estimation of one PU by one thread block (device code).
//
// Integer full search over [-R, R]^2 on channel 0 with SAD + motion cost,
// then quarter-sample refinement with Hadamard SATD + motion cost; the
// definitions are those of xv_motion_search in include/xv.h.
//
// Layout in shared memory:
//   win  u16 [WW][S]    reference window, WW = N + 2R + 8 rows/columns around
//                       the PU (margin R + 4: the 8-tap filter at vectors up
//                       to +-(R + 3/4)), coordinates clamped to the plane when
//                       loaded -- so the search itself never branches on
//                       borders.  Window column c of row y is element
//                       y * S + 4 + c, so the first column of every 8-wide
//                       unit of vectors (c = 8 gx + 4) starts a 16-byte word;
//                       S = 8 (mod 16) spreads the rows of consecutive lanes
//                       over distinct bank groups for 128-bit loads.
//   blk  int32 [N][N]   the PU's channel-0 samples as biased floats (below).
//   scratch             during the integer search: the box-sum table, the
//                       PU's sub-block sums, per-unit bounds, the survivor
//                       list; during refinement: horizontally filtered
//                       columns for the three x-vectors of one stage and the
//                       candidates' row-transformed differences.
// Work split of the integer search: a unit is one candidate row dy and 8
// consecutive dx.  Bound pass: every unit, one lane (or a few) per unit, the
// 8 bounds from 2 x 128-bit table loads per sub-block.  Exact pass: the
// surviving units, P lanes per unit interleaving the block rows; the current
// block's loads are warp-wide broadcasts.  Each lane keeps its best 64-bit
// key (J << 32 | raster index); a block-wide min gives the winner and the
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
    uint32_t exact_cand;   // integer candidates whose SAD was computed exactly
};

__host__ __device__ constexpr int me_win(int N, int R) { return N + 2 * R + 8; }
__host__ __device__ constexpr int me_stride(int N, int R) {
    return (me_win(N, R) + 4 + 7) / 16 * 16 + 8;  // smallest S >= WW + 4 with S % 16 == 8
}

// Exact pruning of the integer search.  For a candidate, split the PU into
// SB x SB sub-blocks; by the triangle inequality the SAD is at least the sum
// over sub-blocks of |sum of current samples - sum of reference samples|.
// A candidate whose bound plus motion cost exceeds the J of a candidate
// already evaluated exactly cannot be the minimum (nor tie with it), so only
// the rest need the exact SAD and the result is that of the full search.
// The reference sums come from a table of SB x SB box sums at every window
// position.  For CTU 16 and 64 it is built and used K row classes at a time
// (box rows y with y - 4 = m mod K, m = 0..K-1): CTU 64 for the whole table
// would not fit next to the window, and at CTU 16 the smaller table keeps
// five blocks per SM resident.
__host__ __device__ constexpr int me_sb(int N) { return N <= 16 ? 4 : (N == 32 ? 8 : 16); }
__host__ __device__ constexpr int me_kcls(int N) { return N == 64 || N == 16 ? 4 : 1; }
__host__ __device__ constexpr int me_side(int R) { return 2 * R + 1; }
__host__ __device__ constexpr bool me_lastcol(int R) { return me_side(R) % 8 == 1; }
// 8-wide column groups of candidates, plus the single last column when
// 2R + 1 = 8m + 1
__host__ __device__ constexpr int me_ngx(int R) { return me_lastcol(R) ? me_side(R) / 8 : (me_side(R) + 7) / 8; }
__host__ __device__ constexpr int me_ngxa(int R) { return me_ngx(R) + (me_lastcol(R) ? 1 : 0); }
__host__ __device__ constexpr int me_units(int R) { return me_side(R) * me_ngxa(R); }
// box-sum table: entries per row (a multiple of 8), row pitch (= 4 mod 32
// words: the rows that 8 consecutive lanes read fall in distinct 16-byte
// bank groups) and rows of one class
__host__ __device__ constexpr int me_tab_stride(int N, int R) { return (8 * me_ngxa(R) + N - me_sb(N) + 7) / 8 * 8; }
__host__ __device__ constexpr int me_tab_pitch(int N, int R) { return (me_tab_stride(N, R) - 4 + 31) / 32 * 32 + 4; }
__host__ __device__ constexpr int me_tab_rows(int N, int R) {
    return (2 * R + N - me_sb(N) + me_kcls(N)) / me_kcls(N);
}

// Byte offsets of the shared-memory regions (every region 16-byte aligned).
// The scratch region holds the pruning tables during the integer search and
// the refinement's filtered columns afterwards.
__host__ __device__ constexpr size_t me_align16(size_t b) { return (b + 15) / 16 * 16; }
// (32 elements of slack after the last row: the box-table build and the
// 8-wide SADs read a few elements past the end of a row)
__host__ __device__ constexpr size_t me_off_blk(int N, int R) {
    return me_align16(((size_t)me_win(N, R) * me_stride(N, R) + 32) * 2);
}
__host__ __device__ constexpr size_t me_off_red(int N, int R) { return me_off_blk(N, R) + me_align16((size_t)N * N * 4); }
__host__ __device__ constexpr size_t me_off_satd(int N, int R) { return me_off_red(N, R) + 64 * 8; }
// motion-cost tables: |se(4d)| for d in [-R, R] (129 at most) and the
// rounded cost of b bits, b < 64
__host__ __device__ constexpr size_t me_off_cost(int N, int R) { return me_off_satd(N, R) + 16 * 4; }
__host__ __device__ constexpr size_t me_off_scr(int N, int R) { return me_off_cost(N, R) + me_align16((129 + 64) * 4); }
// refinement view of the scratch region
__host__ __device__ constexpr size_t me_hp_bytes(int N) { return me_align16((size_t)3 * (N + 8) * N * (N <= 32 ? 4 : 2)); }
__host__ __device__ constexpr size_t me_off_hp(int N, int R) { return me_off_scr(N, R); }
__host__ __device__ constexpr size_t me_off_had(int N, int R) { return me_off_scr(N, R) + me_hp_bytes(N); }
// Candidates' horizontally transformed differences (PUs up to 32 only).
__host__ __device__ constexpr size_t me_had_bytes(int N) { return N <= 32 ? me_align16((size_t)9 * N * N * 2) : 0; }
// pruning view: box table (later the survivor list), sub-block sums of the
// PU, per-unit bounds
__host__ __device__ constexpr size_t me_max(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ constexpr size_t me_tab_bytes(int N, int R) {
    return me_align16(me_max((size_t)me_tab_rows(N, R) * me_tab_pitch(N, R) * 4, (size_t)me_units(R) * 2));
}
__host__ __device__ constexpr size_t me_off_bsub(int N, int R) { return me_off_scr(N, R) + me_tab_bytes(N, R); }
__host__ __device__ constexpr size_t me_off_ulb(int N, int R) {
    return me_off_bsub(N, R) + me_align16((size_t)(N / me_sb(N)) * (N / me_sb(N)) * 4);
}
__host__ __device__ constexpr size_t me_smem_bytes(int N, int R) {
    return me_max(me_off_had(N, R) + me_had_bytes(N), me_off_ulb(N, R) + me_align16((size_t)me_units(R) * 4));
}

// Samples in the window and block are stored as the float 2^23 + v (v <= 1023).
// Its bit pattern is 0x4B000000 | v, so __sad on the raw bits gives |a - b|
// exactly (the bias cancels); read as floats the difference is exact too
// (both operands lie in [2^23, 2^24), where the float spacing is 1).
constexpr int kSampleBias = 0x4B000000;
__device__ __forceinline__ int enc_sample(int v) { return kSampleBias | v; }
__device__ __forceinline__ int dec_sample(int bits) { return bits - kSampleBias; }
// The two 16-bit samples of a word as biased floats' bit patterns, one byte
// permute each: bytes (v.lo, v.hi, 0x00, 0x4B).
__device__ __forceinline__ int enc_lo(uint32_t w) { return (int)__byte_perm(w, (uint32_t)kSampleBias, 0x7410); }
__device__ __forceinline__ int enc_hi(uint32_t w) { return (int)__byte_perm(w, (uint32_t)kSampleBias, 0x7432); }
// 8 window samples (one 16-byte word) as biased values
__device__ __forceinline__ void enc8(const uint16_t* p, int* out) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    out[0] = enc_lo(q.x); out[1] = enc_hi(q.x); out[2] = enc_lo(q.y); out[3] = enc_hi(q.y);
    out[4] = enc_lo(q.z); out[5] = enc_hi(q.z); out[6] = enc_lo(q.w); out[7] = enc_hi(q.w);
}

// Block-wide minimum of v with one barrier: a warp-level minimum, then one
// shared-memory atomicMin per warp into *slot, which must hold ~0 (set
// before an earlier barrier) and is not written again until the caller's
// next item.
__device__ __forceinline__ uint64_t block_min_u64(uint64_t v, uint64_t* slot) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(slot), v);
    __syncthreads();
    return *slot;
}

// SAD of 8 horizontally adjacent candidates over one block row, 8 columns at
// a time: cur[c] against ref[c + k], k = 0..7.  crow: biased int32 samples;
// rrow: window samples, 16-byte aligned.
template <int W>
__device__ __forceinline__ void row_sad8(const int* __restrict__ crow, const uint16_t* __restrict__ rrow,
                                         uint32_t (&sad)[8]) {
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += 8) {
        int cv[8], rv[16];
        {
            const int4 a = *reinterpret_cast<const int4*>(crow + c0);
            const int4 b = *reinterpret_cast<const int4*>(crow + c0 + 4);
            cv[0] = a.x; cv[1] = a.y; cv[2] = a.z; cv[3] = a.w; cv[4] = b.x; cv[5] = b.y; cv[6] = b.z; cv[7] = b.w;
        }
        enc8(rrow + c0, rv);
        enc8(rrow + c0 + 8, rv + 8);
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) sad[k] = __sad(cv[c], rv[c + k], sad[k]);
    }
}

// SAD of one candidate over one block row (the last column of candidates
// when 2R + 1 = 8m + 1); rrow 16-byte aligned.
template <int W>
__device__ __forceinline__ uint32_t row_sad1(const int* __restrict__ crow, const uint16_t* __restrict__ rrow,
                                             uint32_t acc) {
#pragma unroll
    for (int c = 0; c < W; c += 8) {
        int rv[8];
        enc8(rrow + c, rv);
        const int4 a = *reinterpret_cast<const int4*>(crow + c);
        const int4 b = *reinterpret_cast<const int4*>(crow + c + 4);
        acc = __sad(a.x, rv[0], acc); acc = __sad(a.y, rv[1], acc);
        acc = __sad(a.z, rv[2], acc); acc = __sad(a.w, rv[3], acc);
        acc = __sad(b.x, rv[4], acc); acc = __sad(b.y, rv[5], acc);
        acc = __sad(b.z, rv[6], acc); acc = __sad(b.w, rv[7], acc);
    }
    return acc;
}

// Candidate k of a refinement stage around (cx, cy) with step s.  The ring
// of 8 neighbours is taken in raster order (-1,-1), (0,-1), (1,-1), (-1,0),
// (1,0), (-1,1), (0,1), (1,1); with `centre` set, candidate 0 is (cx, cy)
// itself and the ring follows.
__device__ __forceinline__ void stage_cand(int k, int cx, int cy, int s, bool centre, int& mx, int& my) {
    const int r = centre ? k - 1 : k;            // ring index, -1 = the centre
    const int g = r < 0 ? 4 : (r < 4 ? r : r + 1);  // position in the 3 x 3 grid
    mx = cx + (g % 3 - 1) * s;
    my = cy + (g / 3 - 1) * s;
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
// (cx, cy) with step s (candidate k as stage_cand gives it, all within one
// column-set of three x-vectors cx - s, cx, cx + s), SATD summed into satd[].
template <int N, int NT>
__device__ void satd_stage(const uint16_t* __restrict__ wb, int S, int R, const int* __restrict__ blk,
                           int16_t* __restrict__ hp, int cx, int cy, int s, bool centre, int ncand,
                           uint32_t* satd) {
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
        const uint16_t* wr = wb + (rbase + r + R + 4) * S + (x + ix + R + 4);
        int v;
        if (hx == 0) {
            v = wr[0];
        } else {
            int tap[8];
            luma_taps(hx, tap);
            int acc = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) acc += tap[i] * (int)wr[i - 3];
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
        int mvx, mvy;
        stage_cand(k, cx, cy, s, centre, mvx, mvy);
        int j = (mvx - cx) / s + 1;
        int hx = mvx & 3, fy = mvy & 3, iy = mvy >> 2;
        int y = by + lane8;
        const int16_t* col = hp + (size_t)j * (N + 8) * N + bx;
        int r0 = y + iy - 3 - rbase;  // hp row of tap 0
        int d[8];
        int tap[8];
        luma_taps(fy == 0 ? 2 : fy, tap);
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            int v;
            if (fy == 0) {
                int a = col[(r0 + 3) * N + x];
                v = hx == 0 ? a << kShift3 : a;
            } else {
                int acc = 0;
#pragma unroll
                for (int t = 0; t < 8; ++t) acc += tap[t] * (int)col[(r0 + t) * N + x];
                v = hx == 0 ? acc >> kShift1 : acc >> kShift2;
            }
            d[x] = dec_sample(blk[y * N + bx + x]) - wp_round(v);
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

// Refinement stage through shared memory (PUs up to 32): horizontally
// filtered columns, then one task per (candidate, row, 8-column block) that
// forms the 8 predicted samples, their differences and the row Hadamard,
// then one task per (candidate, 8x8 block, column) that finishes the column
// Hadamard; the 8 column tasks of a block are adjacent lanes and add their
// absolute sums before the block's (S + 2) >> 2.
template <int N, int NT>
__device__ void satd_stage_smem(const uint16_t* __restrict__ wb, int S, int R, const int* __restrict__ blk,
                                int* __restrict__ hp, int16_t* __restrict__ had, int cx, int cy, int s,
                                bool centre, int ncand, uint32_t* satd) {
    const int tid = threadIdx.x;
    const int iy_min = (cy - s) >> 2, iy_max = (cy + s) >> 2;
    const int rbase = iy_min - 3;
    const int nr = N + 7 + (iy_max - iy_min);
    for (int idx = tid; idx < 3 * nr * N; idx += NT) {
        int j = idx / (nr * N), rem = idx - j * nr * N;
        int r = rem / N, x = rem - r * N;
        int m = cx + (j - 1) * s;
        int hx = m & 3, ix = m >> 2;
        const uint16_t* wr = wb + (rbase + r + R + 4) * S + (x + ix + R + 4);
        int v;
        if (hx == 0) {
            v = wr[0];
        } else {
            int tap[8];
            luma_taps(hx, tap);
            int acc = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) acc += tap[i] * (int)wr[i - 3];
            v = acc >> kShift1;
        }
        hp[(j * (N + 8) + r) * N + x] = v;
    }
    for (int k = tid; k < ncand; k += NT) satd[k] = 0;
    __syncthreads();
    constexpr int NBX = N / 8;
    for (int task = tid; task < ncand * N * NBX; task += NT) {
        const int k = task / (N * NBX), rem = task - k * N * NBX;
        const int y = rem / NBX, bx = (rem - y * NBX) * 8;
        int mvx, mvy;
        stage_cand(k, cx, cy, s, centre, mvx, mvy);
        const int j = (mvx - cx) / s + 1;
        const int hx = mvx & 3, fy = mvy & 3, iy = mvy >> 2;
        const int* col = hp + (size_t)j * (N + 8) * N + bx;
        const int r0 = y + iy - 3 - rbase;
        int cb[8];
        {
            const int4 a = *reinterpret_cast<const int4*>(blk + y * N + bx);
            const int4 b = *reinterpret_cast<const int4*>(blk + y * N + bx + 4);
            cb[0] = a.x; cb[1] = a.y; cb[2] = a.z; cb[3] = a.w; cb[4] = b.x; cb[5] = b.y; cb[6] = b.z; cb[7] = b.w;
        }
        int d[8];
        if (fy == 0) {
            const int4 a = *reinterpret_cast<const int4*>(col + (r0 + 3) * N);
            const int4 b = *reinterpret_cast<const int4*>(col + (r0 + 3) * N + 4);
            const int v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int x = 0; x < 8; ++x) d[x] = dec_sample(cb[x]) - wp_round(hx == 0 ? v[x] << kShift3 : v[x]);
        } else {
            int tap[8];
            luma_taps(fy, tap);
            const int sh = hx == 0 ? kShift1 : kShift2;
            int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int4 a = *reinterpret_cast<const int4*>(col + (r0 + t) * N);
                const int4 b = *reinterpret_cast<const int4*>(col + (r0 + t) * N + 4);
                acc[0] += tap[t] * a.x; acc[1] += tap[t] * a.y; acc[2] += tap[t] * a.z; acc[3] += tap[t] * a.w;
                acc[4] += tap[t] * b.x; acc[5] += tap[t] * b.y; acc[6] += tap[t] * b.z; acc[7] += tap[t] * b.w;
            }
#pragma unroll
            for (int x = 0; x < 8; ++x) d[x] = dec_sample(cb[x]) - wp_round(acc[x] >> sh);
        }
        hadamard8_row(d);
        uint4 pk;
        pk.x = (uint32_t)(uint16_t)d[0] | ((uint32_t)(uint16_t)d[1] << 16);
        pk.y = (uint32_t)(uint16_t)d[2] | ((uint32_t)(uint16_t)d[3] << 16);
        pk.z = (uint32_t)(uint16_t)d[4] | ((uint32_t)(uint16_t)d[5] << 16);
        pk.w = (uint32_t)(uint16_t)d[6] | ((uint32_t)(uint16_t)d[7] << 16);
        *reinterpret_cast<uint4*>(had + ((size_t)k * N + y) * N + bx) = pk;
    }
    __syncthreads();
    constexpr int NB = NBX * NBX;
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    for (int task = tid; task < ncand * NB * 8; task += NT) {
        const int x = task & 7, kb = task >> 3;
        const int k = kb / NB, b = kb - k * NB;
        const int by = (b / NBX) * 8, bx = (b % NBX) * 8;
        const int16_t* h = had + ((size_t)k * N + by) * N + bx + x;
        int v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = h[i * N];
        hadamard8_row(v);
        int sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) sum += v[i] < 0 ? -v[i] : v[i];
        sum += __shfl_xor_sync(gmask, sum, 1);
        sum += __shfl_xor_sync(gmask, sum, 2);
        sum += __shfl_xor_sync(gmask, sum, 4);
        if (x == 0) atomicAdd(&satd[k], (uint32_t)((sum + 2) >> 2));
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
    uint16_t* win = reinterpret_cast<uint16_t*>(smem);
    const uint16_t* wb = win + 4;  // window column 0 of row 0
    int* blk = reinterpret_cast<int*>(smem + me_off_blk(N, R));
    int16_t* hp = reinterpret_cast<int16_t*>(smem + me_off_hp(N, R));
    uint64_t* red = reinterpret_cast<uint64_t*>(smem + me_off_red(N, R));
    uint32_t* satd = reinterpret_cast<uint32_t*>(smem + me_off_satd(N, R));
    int16_t* had = reinterpret_cast<int16_t*>(smem + me_off_had(N, R));
    int* s_bitsd = reinterpret_cast<int*>(smem + me_off_cost(N, R));  // |se(4d)|, index d + R
    uint32_t* s_costb = reinterpret_cast<uint32_t*>(s_bitsd + 129);    // cost of b bits

    // window with clamped coordinates, 8 samples (16 bytes) per load where the
    // aligned chunk lies inside the plane
    const int wx0 = x0 - R - 4, wy0 = y0 - R - 4;
    const int xa = wx0 - (((wx0 % 8) + 8) % 8);  // 8-aligned start at or left of wx0
    const int nch = (wx0 + WW - xa + 7) / 8;
    const int nwin = WW * nch;
    constexpr int BCH = N / 8;                 // 16-byte chunks per block row
    const int ntask = nwin + N * BCH;          // window chunks, then the PU's
    constexpr int kILP = 5;  // loads in flight per thread before the first store
    for (int base = tid; base < ntask; base += NT * kILP) {
        uint4 v[kILP];
#pragma unroll
        for (int j = 0; j < kILP; ++j) {
            const int task = base + j * NT;
            if (task < nwin) {
                const int r = task / nch, ch = task - r * nch;
                const int yy = min(max(wy0 + r, 0), Hp - 1), xs = xa + 8 * ch;
                const uint16_t* rowp = ref0 + (size_t)yy * Wp;
                if (xs >= 0 && xs + 8 <= Wp) {
                    v[j] = ld_ref16<kCoherent>(reinterpret_cast<const uint4*>(rowp + xs));
                } else {
                    uint32_t w[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        w[i] = (uint32_t)ld_ref<kCoherent>(rowp + min(max(xs + 2 * i, 0), Wp - 1)) |
                               ((uint32_t)ld_ref<kCoherent>(rowp + min(max(xs + 2 * i + 1, 0), Wp - 1)) << 16);
                    v[j] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            } else if (task < ntask) {
                const int t2 = task - nwin, r = t2 / BCH, ch = t2 - r * BCH;
                v[j] = __ldg(reinterpret_cast<const uint4*>(cur0 + (size_t)(y0 + r) * Wp + x0 + 8 * ch));
            }
        }
#pragma unroll
        for (int j = 0; j < kILP; ++j) {
            const int task = base + j * NT;
            const uint32_t w[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
            if (task < nwin) {
                const int r = task / nch, ch = task - r * nch;
                const int c0 = xa + 8 * ch - wx0;
                if (wx0 - xa == 4) {
                    // plane chunk ch is element 8 ch of the row (the columns
                    // outside the window land in the row's padding)
                    *reinterpret_cast<uint4*>(win + r * S + 8 * ch) = v[j];
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int c = c0 + i;
                        if (c >= 0 && c < WW) win[r * S + 4 + c] = (uint16_t)(w[i >> 1] >> (16 * (i & 1)));
                    }
                }
            } else if (task < ntask) {
                const int t2 = task - nwin, r = t2 / BCH, ch = t2 - r * BCH;
                int4 lo, hi;
                lo.x = enc_sample((int)(w[0] & 0xffffu)); lo.y = enc_sample((int)(w[0] >> 16));
                lo.z = enc_sample((int)(w[1] & 0xffffu)); lo.w = enc_sample((int)(w[1] >> 16));
                hi.x = enc_sample((int)(w[2] & 0xffffu)); hi.y = enc_sample((int)(w[2] >> 16));
                hi.z = enc_sample((int)(w[3] & 0xffffu)); hi.w = enc_sample((int)(w[3] >> 16));
                *reinterpret_cast<int4*>(blk + r * N + 8 * ch) = lo;
                *reinterpret_cast<int4*>(blk + r * N + 8 * ch + 4) = hi;
            }
        }
    }
    for (int i = tid; i < 2 * R + 1 + 64; i += NT) {
        if (i < 2 * R + 1) s_bitsd[i] = se_len(4 * (i - R));
        else s_costb[i - (2 * R + 1)] = (uint32_t)((lmv * (int64_t)(i - (2 * R + 1)) + 32768) >> 16);
    }
    {  // sub-block sums and the survivor counts start at 0; the three
       // block-minimum slots at ~0
        int* bs = reinterpret_cast<int*>(smem + me_off_bsub(N, R));
        constexpr int nsb = (N / me_sb(N)) * (N / me_sb(N));
        for (int i = tid; i < nsb + 13; i += NT) {
            if (i < nsb) bs[i] = 0;
            else if (i < nsb + 10) satd[i - nsb] = 0;
            else red[i - nsb - 10] = ~0ull;
        }
    }
    __syncthreads();

    // ---- integer search, exact pruning (see me_sb above)
    // Units: (dy, 8 consecutive dx) for the first 8m columns of candidates;
    // when 2R + 1 = 8m + 1 the last column is a unit of its own (one
    // candidate per dy, column group gx = ngx), else it is covered by an
    // 8-wide unit that discards the candidates beyond R.  Unit u = gx * side
    // + dy + R.
    constexpr int SB = me_sb(N), NS = N / SB, K = me_kcls(N);
    const int side = me_side(R);
    const int ngx = me_ngx(R), ngxa = me_ngxa(R);
    const int units = side * ngxa;
    const int TS = me_tab_stride(N, R), TP = me_tab_pitch(N, R);
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem + me_off_scr(N, R));
    uint16_t* list = reinterpret_cast<uint16_t*>(smem + me_off_scr(N, R));  // after the bounds
    int* bsub = reinterpret_cast<int*>(smem + me_off_bsub(N, R));
    uint32_t* ulb = reinterpret_cast<uint32_t*>(smem + me_off_ulb(N, R));

    // sub-block sums of the PU: one task per (sub-block, row), summing SB
    // biased words (the bias cancels modulo 2^32)
    for (int task = tid; task < NS * NS * SB; task += NT) {
        const int sbk = task / SB, r = task - sbk * SB;
        const int i = sbk / NS, j = sbk - i * NS;
        const int* row = blk + (i * SB + r) * N + j * SB;
        uint32_t acc = 0;
#pragma unroll
        for (int c = 0; c < SB; c += 4) {
            const int4 v = *reinterpret_cast<const int4*>(row + c);
            acc += (uint32_t)v.x + (uint32_t)v.y + (uint32_t)v.z + (uint32_t)v.w;
        }
        atomicAdd(bsub + sbk, (int)(acc - (uint32_t)SB * (uint32_t)kSampleBias));
    }
    // Box table of row class m: entry (t, tx) = sum of the SB x SB window
    // samples with top-left corner (4 + m + K t, 4 + tx).  One task per 8
    // consecutive entries: horizontal running sums over SB window rows (the
    // 16-byte loads start at window column 8 c + 4, a word boundary).
    auto build_tab = [&](int m) {
        const int nr = (2 * R + N - SB - m) / K + 1;
        const int nch = TS / 8;
        for (int task = tid; task < nr * nch; task += NT) {
            const int t = task / nch, c = task - t * nch;
            const uint16_t* w0 = wb + (4 + m + K * t) * S + 8 * c + 4;
            uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 1
            for (int r = 0; r < SB; ++r) {
                uint32_t v[(8 + SB + 7) / 8 * 8];
#pragma unroll
                for (int i = 0; i < 8 + SB; i += 8) {
                    const uint4 q4 = *reinterpret_cast<const uint4*>(w0 + r * S + i);
                    v[i] = q4.x & 0xffffu; v[i + 1] = q4.x >> 16; v[i + 2] = q4.y & 0xffffu; v[i + 3] = q4.y >> 16;
                    v[i + 4] = q4.z & 0xffffu; v[i + 5] = q4.z >> 16; v[i + 6] = q4.w & 0xffffu; v[i + 7] = q4.w >> 16;
                }
                uint32_t h = 0;
#pragma unroll
                for (int i = 0; i < SB; ++i) h += v[i];
                acc[0] += h;
#pragma unroll
                for (int k = 1; k < 8; ++k) {
                    h += v[k + SB - 1] - v[k - 1];
                    acc[k] += h;
                }
            }
            const uint4 o0 = make_uint4(acc[0], acc[1], acc[2], acc[3]);
            const uint4 o1 = make_uint4(acc[4], acc[5], acc[6], acc[7]);
            *reinterpret_cast<uint4*>(tab + t * TP + 8 * c) = o0;
            *reinterpret_cast<uint4*>(tab + t * TP + 8 * c + 4) = o1;
        }
    };
    build_tab(0);
    __syncthreads();

    // bound pass: per unit the smallest bound + motion cost of its valid
    // candidates (dx <= R) into ulb[u]; the unit with the smallest one is the
    // seed
    uint64_t lbbest = ~0ull;
#pragma unroll 1
    for (int m = 0; m < K; ++m) {
        if (m > 0) {
            __syncthreads();
            build_tab(m);
            __syncthreads();
        }
        const int nd = m <= 2 * R ? (2 * R - m) / K + 1 : 0;  // dy + R = m, m + K, ...
        const int ncu = nd * ngxa;
        // lanes per unit: the most (up to NS) that still cover every unit in
        // one round; one when even that is impossible (latency: a single
        // lane per unit needs no reduction and no shared epilogue)
        int P = 1;
        while (2 * P <= NS && ncu * 2 * P <= NT) P *= 2;
        const int q = tid & (P - 1);
        const unsigned pmask = P == 1 ? 0u : ((1u << P) - 1u) << ((threadIdx.x & 31) & ~(P - 1));
        for (int v = tid / P; v < ncu; v += NT / P) {
            const int gx = v / nd;
            const int dyi = m + K * (v - gx * nd);
            const uint32_t* trow = tab + ((dyi - m) / K) * TP + 8 * gx;
            uint32_t lb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = q; i < NS; i += P) {
                const uint32_t* tr = trow + i * (SB / K) * TP;
#pragma unroll
                for (int j = 0; j < NS; ++j) {
                    const uint4 b0 = *reinterpret_cast<const uint4*>(tr + SB * j);
                    const uint4 b1 = *reinterpret_cast<const uint4*>(tr + SB * j + 4);
                    const int cs = bsub[i * NS + j];
                    lb[0] = __sad(cs, (int)b0.x, lb[0]); lb[1] = __sad(cs, (int)b0.y, lb[1]);
                    lb[2] = __sad(cs, (int)b0.z, lb[2]); lb[3] = __sad(cs, (int)b0.w, lb[3]);
                    lb[4] = __sad(cs, (int)b1.x, lb[4]); lb[5] = __sad(cs, (int)b1.y, lb[5]);
                    lb[6] = __sad(cs, (int)b1.z, lb[6]); lb[7] = __sad(cs, (int)b1.w, lb[7]);
                }
            }
            for (int o = 1; o < P; o <<= 1)
#pragma unroll
                for (int k = 0; k < 8; ++k) lb[k] += __shfl_xor_sync(pmask, lb[k], o);
            if (q == 0) {
                const int by = s_bitsd[dyi];
                uint32_t mn = ~0u;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int dx = gx * 8 - R + k;
                    if (dx <= R) {
                        const uint32_t J = lb[k] + s_costb[s_bitsd[dx + R] + by];
                        mn = J < mn ? J : mn;
                    }
                }
                const int u = gx * side + dyi;
                ulb[u] = mn;
                const uint64_t key = ((uint64_t)mn << 32) | (uint32_t)u;
                lbbest = key < lbbest ? key : lbbest;
            }
        }
    }
    lbbest = block_min_u64(lbbest, red);  // its barrier also ends the bound pass
    const int useed = (int)(lbbest & 0xffffffffu);

    // Exact search in two rounds of the same code: round 0 the seed unit alone
    // (its best J is the pruning threshold), round 1 the surviving units; P
    // lanes per unit interleave the block rows.
    uint64_t best = ~0ull;
    int M = 1;
    uint32_t exact_cand = 0;
#pragma unroll 1
    for (int round = 0; round < 2; ++round) {
        if (round == 1) {
            best = block_min_u64(best, red + 2);  // the seed unit's best key, on every thread
            const uint32_t thr = (uint32_t)(best >> 32);
            // survivors: units (other than the seed) whose bound does not exceed
            // the seed's J; warp-aggregated appends (satd[9] counts the single-column
            // ones, for the executed-work statistic)
            {
                const int lane = threadIdx.x & 31;
                for (int u0 = tid - lane; u0 < units; u0 += NT) {
                    const int u = u0 + lane;
                    const bool keep = u < units && u != useed && ulb[u] <= thr;
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    if (!bal) continue;
                    const unsigned bal1 = __ballot_sync(0xffffffffu, keep && u >= ngx * side);
                    unsigned base = 0;
                    if (lane == 0) {
                        base = atomicAdd(satd + 8, (uint32_t)__popc(bal));
                        if (bal1) atomicAdd(satd + 9, (uint32_t)__popc(bal1));
                    }
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (keep) list[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)u;
                }
            }
            __syncthreads();
            M = (int)satd[8];
            exact_cand = 8u * (uint32_t)(M - (int)satd[9]) + satd[9] + (useed >= ngx * side ? 1u : 8u);
        }
        {
            int P = 1;
            while (P < 32 && 2 * P <= N && M * 2 * P <= NT) P *= 2;
            const int q = tid & (P - 1);
            const unsigned pmask = P == 1 ? 0u : (P == 32 ? 0xffffffffu : ((1u << P) - 1u) << ((threadIdx.x & 31) & ~(P - 1)));
            for (int i = tid / P; i < M; i += NT / P) {
                const int u = round == 0 ? useed : (int)list[i];
                const int gx = u / side, dyi = u - gx * side;
                const int dx0 = gx * 8 - R;
                const int woff = (dyi + 4) * S + gx * 8 + 4;
                const uint32_t rowbase = (uint32_t)(dyi * side);
                const int by = s_bitsd[dyi];
                if (gx == ngx) {  // the single last column, dx = R
                    uint32_t sad1 = 0;
                    for (int r = q; r < N; r += P) sad1 = row_sad1<N>(blk + r * N, wb + woff + r * S, sad1);
                    for (int o = 1; o < P; o <<= 1) sad1 += __shfl_xor_sync(pmask, sad1, o);
                    if (q == 0) {
                        const uint32_t J = sad1 + s_costb[s_bitsd[2 * R] + by];
                        const uint64_t key = ((uint64_t)J << 32) | (rowbase + (uint32_t)(2 * R));
                        best = key < best ? key : best;
                    }
                    continue;
                }
                uint32_t sad[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                // one row at a time (a second, FP32-pipe copy of the row code for
                // a third of the rows measured slower: it costs more in code size
                // than it gains in pipe balance, the survivors being few)
#pragma unroll 1
                for (int r = q; r < N; r += P) row_sad8<N>(blk + r * N, wb + woff + r * S, sad);
                for (int o = 1; o < P; o <<= 1)
#pragma unroll
                    for (int k = 0; k < 8; ++k) sad[k] += __shfl_xor_sync(pmask, sad[k], o);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int dx = dx0 + k;
                    if ((k & (P - 1)) == q && dx <= R) {  // the P lanes share the candidates
                        const uint32_t J = sad[k] + s_costb[s_bitsd[dx + R] + by];
                        const uint64_t key = ((uint64_t)J << 32) | (rowbase + (uint32_t)(dx + R));
                        best = key < best ? key : best;
                    }
                }
            }
        }
    }
    best = block_min_u64(best, red + 1);
    MeResult res;
    {
        int idx = (int)(best & 0xffffffffu);
        res.mvy_int = idx / side - R;
        res.mvx_int = idx - (idx / side) * side - R;
        res.cost_int = (uint32_t)(best >> 32);
        res.exact_cand = exact_cand;
    }

    // ---- quarter-sample refinement: centre + 8 half-sample, then 8 quarter
    int cx = 4 * res.mvx_int, cy = 4 * res.mvy_int;
    if constexpr (N <= 32)
        satd_stage_smem<N, NT>(wb, S, R, blk, reinterpret_cast<int*>(hp), had, cx, cy, 2, true, 9, satd);
    else satd_stage<N, NT>(wb, S, R, blk, hp, cx, cy, 2, true, 9, satd);
    uint32_t bJ = satd[0] + mv_cost(cx, cy, lmv);
    int bx = cx, by = cy;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        int mx, my;
        stage_cand(k, cx, cy, 2, true, mx, my);
        const uint32_t J = satd[k] + mv_cost(mx, my, lmv);
        if (J < bJ) { bJ = J; bx = mx; by = my; }
    }
    __syncthreads();
    cx = bx; cy = by;
    if constexpr (N <= 32)
        satd_stage_smem<N, NT>(wb, S, R, blk, reinterpret_cast<int*>(hp), had, cx, cy, 1, false, 8, satd);
    else satd_stage<N, NT>(wb, S, R, blk, hp, cx, cy, 1, false, 8, satd);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int mx, my;
        stage_cand(k, cx, cy, 1, false, mx, my);
        const uint32_t J = satd[k] + mv_cost(mx, my, lmv);
        if (J < bJ) { bJ = J; bx = mx; by = my; }
    }
    __syncthreads();
    res.mvx = bx;
    res.mvy = by;
    res.cost = bJ;
    return res;
}

}  // namespace xvd
