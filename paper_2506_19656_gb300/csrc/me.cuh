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
#include "../../include/xv.h"
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
// (box rows y with y - 4 = m mod K, m = 0..K-1) by default: at CTU 64 the
// whole table would not fit next to the window (two classes do, up to 178 KB
// at R = 64, and measured 13 % faster than four), and at CTU 16 four classes
// keep five blocks per SM resident in the persistent kernel.  The per-frame
// search at CTU 16 builds the whole table at once where it fits (me_pu's KC):
// one build and one bound pass instead of four of each.
__host__ __device__ constexpr int me_sb(int N) { return N <= 16 ? 4 : (N == 32 ? 8 : 16); }
__host__ __device__ constexpr int me_kcls(int N) { return N == 64 ? 2 : (N == 16 ? 4 : 1); }
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
__host__ __device__ constexpr int me_tab_rows(int N, int R, int K) { return (2 * R + N - me_sb(N) + K) / K; }

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
// refinement view of the scratch region: three horizontally filtered planes
// (int16 [N + 8][N] each: block rows -4 .. N + 3 around the integer vector)
__host__ __device__ constexpr size_t me_plane_elems(int N) { return (size_t)(N + 8) * N; }
__host__ __device__ constexpr size_t me_planes_bytes(int N) { return me_align16(3 * me_plane_elems(N) * 2); }
// pruning view: box table (later the survivor list), sub-block sums of the
// PU, per-unit bounds
__host__ __device__ constexpr size_t me_max(size_t a, size_t b) { return a > b ? a : b; }
// (K = the box table's row classes; the two-argument forms take me_kcls(N))
__host__ __device__ constexpr size_t me_tab_bytes(int N, int R, int K) {
    return me_align16(me_max((size_t)me_tab_rows(N, R, K) * me_tab_pitch(N, R) * 4, (size_t)me_units(R) * 2));
}
__host__ __device__ constexpr size_t me_off_bsub(int N, int R, int K) { return me_off_scr(N, R) + me_tab_bytes(N, R, K); }
__host__ __device__ constexpr size_t me_off_ulb(int N, int R, int K) {
    return me_off_bsub(N, R, K) + me_align16((size_t)(N / me_sb(N)) * (N / me_sb(N)) * 4);
}
__host__ __device__ constexpr size_t me_smem_bytes(int N, int R, int K) {
    return me_max(me_off_scr(N, R) + me_planes_bytes(N), me_off_ulb(N, R, K) + me_align16((size_t)me_units(R) * 4));
}
__host__ __device__ constexpr size_t me_smem_bytes(int N, int R) { return me_smem_bytes(N, R, me_kcls(N)); }

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

// Horizontal pass of the refinement for up to three x-vectors m[i] (quarter
// samples) into planes dst[i] (int16 [N + 8][N]): row r holds block row
// q = r - 4 + my, column x the sample at x + m/4: the full sample itself
// when m is a multiple of 4, else the 8-tap filter of its phase over the
// window, >> shift1.  One task per plane row and 8 columns: 15 window
// samples in registers give the 8 outputs, stored as one 16-byte word.
template <int N, int NT>
__device__ __forceinline__ void refine_planes(const uint16_t* __restrict__ wb, int S, int R, int my, int np,
                                              int m0, int m1, int m2, int16_t* d0, int16_t* d1, int16_t* d2) {
    constexpr int SPR = N / 8;
    constexpr int TPP = (N + 8) * SPR;
    for (int task = threadIdx.x; task < np * TPP; task += NT) {
        const int pi = task / TPP, rem = task - pi * TPP;
        const int r = rem / SPR, x0 = (rem - r * SPR) * 8;
        const int m = pi == 0 ? m0 : (pi == 1 ? m1 : m2);
        int16_t* dst = pi == 0 ? d0 : (pi == 1 ? d1 : d2);
        const int hx = m & 3, ix = m >> 2;
        const uint16_t* w = wb + (r + my + R) * S + x0 + ix + R + 4;  // block row q, column x0 + ix
        int o[8];
        if (hx == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c) o[c] = w[c];
        } else {
            int v[15];
#pragma unroll
            for (int i = 0; i < 15; ++i) v[i] = w[i - 3];
            int tap[8];
            luma_taps(hx, tap);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                int acc = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) acc += tap[i] * v[c + i];
                o[c] = acc >> kShift1;
            }
        }
        uint4 pk;
        pk.x = (uint32_t)(uint16_t)o[0] | ((uint32_t)(uint16_t)o[1] << 16);
        pk.y = (uint32_t)(uint16_t)o[2] | ((uint32_t)(uint16_t)o[3] << 16);
        pk.z = (uint32_t)(uint16_t)o[4] | ((uint32_t)(uint16_t)o[5] << 16);
        pk.w = (uint32_t)(uint16_t)o[6] | ((uint32_t)(uint16_t)o[7] << 16);
        *reinterpret_cast<uint4*>(dst + r * N + x0) = pk;
    }
}

// 8 int16 of a plane row (16-byte aligned) as ints.
__device__ __forceinline__ void load_row8(const int16_t* p, int (&v)[8]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[2 * i] = (int)(int16_t)(w[i] & 0xffffu);
        v[2 * i + 1] = (int)w[i] >> 16;
    }
}

// W (1, 2 or 4) int16 of a plane row (2W-byte aligned) as ints.
template <int W>
__device__ __forceinline__ void load_row_n(const int16_t* p, int (&v)[W]) {
    if constexpr (W == 4) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = (int)(int16_t)(q.x & 0xffffu); v[1] = (int)q.x >> 16;
        v[2] = (int)(int16_t)(q.y & 0xffffu); v[3] = (int)q.y >> 16;
    } else if constexpr (W == 2) {
        const uint32_t q = *reinterpret_cast<const uint32_t*>(p);
        v[0] = (int)(int16_t)(q & 0xffffu); v[1] = (int)q >> 16;
    } else {
        v[0] = p[0];
    }
}

// Part of the SATD of the 8x8 block at (bx0, by0) of the PU, against its
// prediction at a quarter-sample vector whose horizontal pass is plane P
// (vertical phase fy, iyr = the vector's integer row - my, hx0 = its column
// is a full sample): LPB lanes (2, 4 or 8, adjacent, all calling this for the
// same block) take 8 / LPB columns each, lane part p the columns from
// bx0 + (8 / LPB) p.  The prediction (vertical 8-tap filter over 15 plane
// rows, or the plane row itself; default weighted rounding), the difference
// with the current block and the Hadamard transform along the columns stay
// in the lane's registers; the transform along the rows takes its stages
// across the lanes by shuffle and the rest within the lane (the Hadamard's
// stages commute, and the absolute sum does not depend on the order of the
// coefficients).  Every lane of the group returns the block's (S + 2) >> 2.
template <int N, int LPB>
__device__ __forceinline__ uint32_t satd_part(const int16_t* __restrict__ P, const int* __restrict__ blk, int bx0,
                                              int by0, int part, int iyr, int fy, bool hx0) {
    constexpr int CW = 8 / LPB;
    constexpr int LCW = CW == 4 ? 2 : (CW == 2 ? 1 : 0);
    const int xc = bx0 + CW * part;
    int a[8][CW];
    if (fy == 0) {
        const int16_t* p = P + (by0 + iyr + 4) * N + xc;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            int v[CW];
            load_row_n<CW>(p + y * N, v);
#pragma unroll
            for (int c = 0; c < CW; ++c) a[y][c] = hx0 ? v[c] : wp_round(v[c]);
        }
    } else {
        int tap[8];
        luma_taps(fy, tap);
#pragma unroll
        for (int y = 0; y < 8; ++y)
#pragma unroll
            for (int c = 0; c < CW; ++c) a[y][c] = 0;
        const int16_t* p = P + (by0 + iyr + 1) * N + xc;  // block row by0 + iy - 3
#pragma unroll
        for (int rho = 0; rho < 15; ++rho) {
            int v[CW];
            load_row_n<CW>(p + rho * N, v);
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                const int t = rho - y;
                if (t >= 0 && t < 8)
#pragma unroll
                    for (int c = 0; c < CW; ++c) a[y][c] += tap[t] * v[c];
            }
        }
        const int sh = hx0 ? kShift1 : kShift2;
#pragma unroll
        for (int y = 0; y < 8; ++y)
#pragma unroll
            for (int c = 0; c < CW; ++c) a[y][c] = wp_round(a[y][c] >> sh);
    }
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int* cp = blk + (by0 + y) * N + xc;
#pragma unroll
        for (int c = 0; c < CW; ++c) a[y][c] = dec_sample(cp[c]) - a[y][c];
    }
    // Hadamard along each column (over y)
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        int col[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) col[y] = a[y][c];
        hadamard8_row(col);
#pragma unroll
        for (int y = 0; y < 8; ++y) a[y][c] = col[y];
    }
    // along each row: the stages over the column-index bits held by the
    // lane part (across lanes), then those within the lane
    const unsigned gmask = ((1u << LPB) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(LPB - 1));
#pragma unroll
    for (int hl = 1; hl < LPB; hl <<= 1) {
        const bool upper = (part & hl) != 0;
#pragma unroll
        for (int y = 0; y < 8; ++y)
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                const int o = __shfl_xor_sync(gmask, a[y][c], hl);
                a[y][c] = upper ? o - a[y][c] : a[y][c] + o;
            }
    }
    uint32_t sum = 0;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
#pragma unroll
        for (int h = 1; h < CW; h <<= 1)
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (!(c & h)) {
                    const int u = a[y][c], w = a[y][c + h];
                    a[y][c] = u + w;
                    a[y][c + h] = u - w;
                }
#pragma unroll
        for (int c = 0; c < CW; ++c) sum += (uint32_t)abs(a[y][c]);
    }
#pragma unroll
    for (int hl = 1; hl < LPB; hl <<= 1) sum += __shfl_xor_sync(gmask, sum, hl);
    (void)LCW;
    return (sum + 2) >> 2;
}

// Lanes per 8x8 block of the refinement's SATD: more for small PUs, which
// have few blocks per candidate.
template <int N>
__host__ __device__ constexpr int me_lpb() { return N >= 32 ? 2 : 8; }

// The search window by one tiled bulk copy (TMA): thread 0 initialises the
// item's mbarrier, announces the copy's bytes and issues it; the copy lands
// while the block loads the PU's samples and the cost tables.  `tmap` is a
// 3-D tensor map (x, y, group) over the reference frame's channel-0 planes
// (a kernel parameter), box (S, WW, 1), read from chunk column xa and row
// wy0 of group tz.
__device__ __forceinline__ void window_tma_issue(uint16_t* win, const void* tmap, int xa, int wy0, int tz,
                                                 uint32_t mbar, uint32_t bytes) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(win);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // earlier reads of the window (the previous item) before the copy engine's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(tmap), "r"(xa), "r"(wy0), "r"(tz), "r"(mbar)
        : "memory");
}

// Waits (bounded) for the mbarrier's phase `parity` to complete; false when
// the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long polls) {
    for (long long i = 0; i < polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Motion estimation of the PU at (x0, y0).  cur0/ref0: channel-0 planes.
// Must be called by all NT threads of the block; smem holds
// me_smem_bytes(N, R, KC) (KC: the box table's row classes, see me_kcls).
// With `tmap` (a tensor map over the reference planes, see window_tma_issue;
// tz = the group's coordinate in it) the window comes by TMA where it lies
// inside the plane; a copy that does not complete within the wait bound sets
// *err to XV_ETIMEOUT (the result is then not valid).
template <int N, int NT, bool kCoherent = false, int KC = me_kcls(N)>
__device__ MeResult me_pu(const uint16_t* __restrict__ cur0, const uint16_t* __restrict__ ref0,
                          int Hp, int Wp, int x0, int y0, int R, int64_t lmv, unsigned char* smem,
                          const void* tmap = nullptr, int tz = 0, int* err = nullptr,
                          long long tma_polls = 1ll << 24) {
    static_assert(N % 8 == 0, "PU size must be a multiple of 8");
    const int tid = threadIdx.x;
    const int WW = me_win(N, R), S = me_stride(N, R);
    uint16_t* win = reinterpret_cast<uint16_t*>(smem);
    const uint16_t* wb = win + 4;  // window column 0 of row 0
    int* blk = reinterpret_cast<int*>(smem + me_off_blk(N, R));
    int16_t* planes = reinterpret_cast<int16_t*>(smem + me_off_scr(N, R));
    uint64_t* red = reinterpret_cast<uint64_t*>(smem + me_off_red(N, R));
    uint32_t* satd = reinterpret_cast<uint32_t*>(smem + me_off_satd(N, R));
    int* s_bitsd = reinterpret_cast<int*>(smem + me_off_cost(N, R));  // |se(4d)|, index d + R
    uint32_t* s_costb = reinterpret_cast<uint32_t*>(s_bitsd + 129);    // cost of b bits

    // window with clamped coordinates, 8 samples (16 bytes) per load where the
    // aligned chunk lies inside the plane
    const int wx0 = x0 - R - 4, wy0 = y0 - R - 4;
    const int xa = wx0 - (((wx0 % 8) + 8) % 8);  // 8-aligned start at or left of wx0
    const int nch = (wx0 + WW - xa + 7) / 8;
    // the TMA path: the window (from chunk column xa, S columns) inside the
    // plane, starting 4 samples into its chunk as the layout wants
    const bool tma = tmap != nullptr && wx0 - xa == 4 && xa >= 0 && xa + S <= Wp && wy0 >= 0 && wy0 + WW <= Hp;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(red + 16);
    if (tma && tid == 0) window_tma_issue(win, tmap, xa, wy0, tz, mbar, (uint32_t)(S * WW * 2));
    const int nwin = tma ? 0 : WW * nch;
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
        int* bs = reinterpret_cast<int*>(smem + me_off_bsub(N, R, KC));
        constexpr int nsb = (N / me_sb(N)) * (N / me_sb(N));
        for (int i = tid; i < nsb + 13; i += NT) {
            if (i < nsb) bs[i] = 0;
            else if (i < nsb + 10) satd[i - nsb] = 0;
            else red[i - nsb - 10] = ~0ull;
        }
    }
    __syncthreads();
    if (tma && !mbar_wait_bounded(mbar, 0, tma_polls)) {
        if (err) atomicExch(err, (int)XV_ETIMEOUT);
        mbar_wait_bounded(mbar, 0, 1ll << 24);  // give the copy in flight a second bound before the smem is reused
    }

    // ---- integer search, exact pruning (see me_sb above)
    // Units: (dy, 8 consecutive dx) for the first 8m columns of candidates;
    // when 2R + 1 = 8m + 1 the last column is a unit of its own (one
    // candidate per dy, column group gx = ngx), else it is covered by an
    // 8-wide unit that discards the candidates beyond R.  Unit u = gx * side
    // + dy + R.
    constexpr int SB = me_sb(N), NS = N / SB, K = KC;
    static_assert(SB % K == 0, "row classes divide the sub-block side");
    const int side = me_side(R);
    const int ngx = me_ngx(R), ngxa = me_ngxa(R);
    const int units = side * ngxa;
    const int TS = me_tab_stride(N, R), TP = me_tab_pitch(N, R);
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem + me_off_scr(N, R));
    uint16_t* list = reinterpret_cast<uint16_t*>(smem + me_off_scr(N, R));  // after the bounds
    int* bsub = reinterpret_cast<int*>(smem + me_off_bsub(N, R, KC));
    uint32_t* ulb = reinterpret_cast<uint32_t*>(smem + me_off_ulb(N, R, KC));

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
    // samples with top-left corner (4 + m + K t, 4 + tx).  One task per MR
    // consecutive table rows and 8 consecutive entries (16-byte loads start
    // at window column 8 c + 4, a word boundary): the column sums over SB
    // window rows are kept as packed 16-bit pairs (SB x 1023 < 2^16, so a
    // lane never carries into the next, and a row leaves a sum only after it
    // entered it) and slid down K rows from one table row to the next; the
    // 8 entries are sliding sums of SB column sums.
    auto build_tab = [&](int m) {
        constexpr int MR = 4;
        constexpr int NQ = (8 + SB + 7) / 8;  // 16-byte loads per row segment
        const int nr = (2 * R + N - SB - m) / K + 1;
        const int nch = TS / 8;
        const int ngrp = (nr + MR - 1) / MR;
        for (int task = tid; task < ngrp * nch; task += NT) {
            const int g = task / nch, c = task - g * nch;
            const int t0 = g * MR;
            const uint16_t* w0 = wb + (4 + m + K * t0) * S + 8 * c + 4;
            uint32_t vs[4 * NQ];
#pragma unroll
            for (int i = 0; i < 4 * NQ; ++i) vs[i] = 0u;
#pragma unroll 4
            for (int r = 0; r < SB; ++r) {
#pragma unroll
                for (int j = 0; j < NQ; ++j) {
                    const uint4 q4 = *reinterpret_cast<const uint4*>(w0 + r * S + 8 * j);
                    vs[4 * j] += q4.x; vs[4 * j + 1] += q4.y; vs[4 * j + 2] += q4.z; vs[4 * j + 3] += q4.w;
                }
            }
#pragma unroll 1
            for (int tt = 0; tt < MR; ++tt) {
                const int t = t0 + tt;
                if (t >= nr) break;
                if (tt > 0) {
#pragma unroll 1
                    for (int r = K * (tt - 1); r < K * tt; ++r) {
#pragma unroll
                        for (int j = 0; j < NQ; ++j) {
                            const uint4 a4 = *reinterpret_cast<const uint4*>(w0 + (r + SB) * S + 8 * j);
                            const uint4 d4 = *reinterpret_cast<const uint4*>(w0 + r * S + 8 * j);
                            vs[4 * j] += a4.x - d4.x; vs[4 * j + 1] += a4.y - d4.y;
                            vs[4 * j + 2] += a4.z - d4.z; vs[4 * j + 3] += a4.w - d4.w;
                        }
                    }
                }
                uint32_t v[8 * NQ];
#pragma unroll
                for (int i = 0; i < 4 * NQ; ++i) { v[2 * i] = vs[i] & 0xffffu; v[2 * i + 1] = vs[i] >> 16; }
                uint32_t acc[8];
                uint32_t h = 0;
#pragma unroll
                for (int i = 0; i < SB; ++i) h += v[i];
                acc[0] = h;
#pragma unroll
                for (int k = 1; k < 8; ++k) {
                    h += v[k + SB - 1] - v[k - 1];
                    acc[k] = h;
                }
                *reinterpret_cast<uint4*>(tab + t * TP + 8 * c) = make_uint4(acc[0], acc[1], acc[2], acc[3]);
                *reinterpret_cast<uint4*>(tab + t * TP + 8 * c + 4) = make_uint4(acc[4], acc[5], acc[6], acc[7]);
            }
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
    // Stage 1 evaluates the centre (the integer vector) and its 8 half-sample
    // neighbours, stage 2 the 8 quarter-sample neighbours of the best; each
    // candidate's J = SATD + motion cost replaces the best only when strictly
    // lower, in the ring order.  A stage builds the horizontal passes of its
    // three x-vectors (stage 2 keeps the one of the best's column from stage
    // 1), then one task per (candidate, 8x8 block) forms the prediction and
    // the SATD.
    constexpr int NB = (N / 8) * (N / 8);
    const int my = res.mvy_int;
    int16_t* const pl0 = planes;
    int16_t* const pl1 = planes + me_plane_elems(N);
    int16_t* const pl2 = planes + 2 * me_plane_elems(N);
    int cx = 4 * res.mvx_int, cy = 4 * my;
    int bx = cx, by = cy;
    uint32_t bJ = 0;
    int pm0 = cx - 2, pm1 = cx, pm2 = cx + 2;  // x-vector of each plane
#pragma unroll 1
    for (int stage = 0; stage < 2; ++stage) {
        const int s = stage == 0 ? 2 : 1;
        const int ncand = stage == 0 ? 9 : 8;
        if (stage == 0) {
            refine_planes<N, NT>(wb, S, R, my, 3, pm0, pm1, pm2, pl0, pl1, pl2);
        } else {
            // keep the plane of the best's column; the other two take bx - 1 and bx + 1
            if (pm0 == bx) {
                pm1 = bx - 1; pm2 = bx + 1;
                refine_planes<N, NT>(wb, S, R, my, 2, pm1, pm2, 0, pl1, pl2, nullptr);
            } else if (pm1 == bx) {
                pm0 = bx - 1; pm2 = bx + 1;
                refine_planes<N, NT>(wb, S, R, my, 2, pm0, pm2, 0, pl0, pl2, nullptr);
            } else {
                pm0 = bx - 1; pm1 = bx + 1;
                refine_planes<N, NT>(wb, S, R, my, 2, pm0, pm1, 0, pl0, pl1, nullptr);
            }
        }
        // stage 2 sums into its own array, so that stage 1's selection
        // needs no barrier before stage 2 starts
        uint32_t* acc = stage == 0 ? satd : reinterpret_cast<uint32_t*>(red + 4);
        for (int k = tid; k < ncand; k += NT) acc[k] = 0;
        __syncthreads();
        // LPB adjacent lanes per (candidate, 8x8 block); NT is a multiple of
        // 32, so all lanes of a block are taken in the same round
        constexpr int LPB = me_lpb<N>();
        for (int task = tid; task < LPB * ncand * NB; task += NT) {
            const int kb = task / LPB;
            // stage 1 takes the centre last: without a vertical filter it is
            // the cheapest candidate, so the tasks past the first round are
            // short ones
            const int kk = kb / NB, b = kb - kk * NB;
            const int k = stage == 0 ? (kk + 1) % 9 : kk;
            int mvx, mvy;
            stage_cand(k, cx, cy, s, stage == 0, mvx, mvy);
            const int16_t* P = pm0 == mvx ? pl0 : (pm1 == mvx ? pl1 : pl2);
            const uint32_t v = satd_part<N, LPB>(P, blk, (b % (N / 8)) * 8, (b / (N / 8)) * 8, task & (LPB - 1),
                                                 (mvy >> 2) - my, mvy & 3, (mvx & 3) == 0);
            if ((task & (LPB - 1)) == 0) atomicAdd(&acc[k], v);
        }
        __syncthreads();
        int k0 = 0;
        if (stage == 0) { bJ = acc[0] + mv_cost(cx, cy, lmv); k0 = 1; }
#pragma unroll 1
        for (int k = k0; k < ncand; ++k) {
            int mx, my2;
            stage_cand(k, cx, cy, s, stage == 0, mx, my2);
            const uint32_t J = acc[k] + mv_cost(mx, my2, lmv);
            if (J < bJ) { bJ = J; bx = mx; by = my2; }
        }
        if (stage == 1) __syncthreads();  // the caller may reuse the shared memory
        cx = bx;
        cy = by;
    }
    res.mvx = bx;
    res.mvy = by;
    res.cost = bJ;
    return res;
}

}  // namespace xvd
