// tqr.cuh -- transform, quantise, reconstruct one CU by one thread block.
//
// Definitions: xv_transform_quant_recon in include/xv.h.  For each allowed
// TU size (ascending) the whole CU goes through
//   rows:    Y = rs(X T^T, log2N + 1)             one thread per TU row
//   columns: C = rs(T Y, log2N + 6), quantise, dequantise,
//            E = clip16(rs(T^T D, 7))             one thread per TU column
//   rows:    r = rs(E T, 10), recon = clip(pred + r)
// and the size with the least (SSE << 8) + lambda * bits is kept (ties to the
// larger).  The kept size's reconstruction and levels are copied out as soon
// as a size improves on the best so far, so no second buffer set is needed.
//
// Shared memory (all [3][N][N] unless noted):
//   cur u16, pred u16, work int16 (Y, then E), lev int16, rec u16,
//   stage int16 [3][N+7][N+7] (the motion-compensation windows),
//   hbuf int16 [3][N+7][N] (their horizontal pass), reductions.
#pragma once
#include <cstdint>
#include "xv_dev.cuh"

namespace xvd {

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }
// The motion-compensation window of a channel (N + 7 rows and columns) is
// staged as whole 16-byte chunks of the reference rows: its first column
// lies anywhere in an 8-sample chunk, so a staged row holds up to
// (N + 7 + 7) / 8 + 1 chunks.
__host__ __device__ constexpr int tqr_stage_stride(int N) { return ((N + 7 + 7) / 8 + 1) * 8; }
__host__ __device__ constexpr size_t tqr_stage_bytes(int N) { return align16((size_t)3 * (N + 7) * tqr_stage_stride(N) * 2); }
__host__ __device__ constexpr size_t tqr_hbuf_bytes(int N) { return align16((size_t)3 * (N + 7) * N * 2); }
// Byte offsets of the shared-memory regions (every region 16-byte aligned).
__host__ __device__ constexpr size_t tqr_off_stage(int N) { return align16((size_t)5 * 3 * N * N * 2); }
__host__ __device__ constexpr size_t tqr_off_hbuf(int N) { return tqr_off_stage(N) + tqr_stage_bytes(N); }
__host__ __device__ constexpr size_t tqr_off_red(int N) { return tqr_off_hbuf(N) + tqr_hbuf_bytes(N); }
// the 32-point halves' coefficient table (CUs of 32 and more)
__host__ __device__ constexpr size_t tqr_off_t32(int N) { return tqr_off_red(N) + 64 * 8; }
__host__ __device__ constexpr size_t tqr_seq_smem_bytes(int N) {
    return tqr_off_t32(N) + (N >= 32 ? (size_t)kT32HalvesInts * 4 : 0);
}

// Block-wide sums of (a, b) with one barrier: a warp-level sum, then one
// shared-memory atomic per warp into slot `slot` of red (red[slot] for a,
// the 32-bit word 8 + slot of red for b), which must hold 0 (cleared before
// an earlier barrier) and is not reused within the CU.
template <int NT>
__device__ __forceinline__ void block_sum2_slot(uint64_t& a, uint32_t& b, uint64_t* red, int slot) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    uint32_t* rb = reinterpret_cast<uint32_t*>(red) + 8;
    if ((threadIdx.x & 31) == 0 && (a | b)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(red + slot), (unsigned long long)a);
        atomicAdd(rb + slot, b);
    }
    __syncthreads();
    a = red[slot];
    b = rb[slot];
}

template <int NT>
__device__ __forceinline__ void block_sum2(uint64_t& a, uint32_t& b, uint64_t* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { red[warp] = a; red[32 + warp] = b; }
    __syncthreads();
    a = 0; b = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) { a += red[w]; b += (uint32_t)red[32 + w]; }
    __syncthreads();
}

// Loads the CU's current samples (s_cur) and, with a reference, the motion-
// compensation windows of all three channels (rows y0+iy-3 .. y0+iy+N+3,
// columns likewise, coordinates clamped to the plane) as whole 16-byte
// chunks of the reference rows into s_stage [3][N+7][tqr_stage_stride(N)]
// (window column q at staged column q + off, off = the window's offset in
// its first chunk), every load of a thread in flight before its stores.
// Then predicts the CU (s_pred; flat 512 without a reference): HEVC 8-tap
// luma filter, horizontal pass into s_hbuf [3][N+7][N] (one task per 8
// outputs of a row, its 15 inputs in registers), vertical pass over 4 x 4
// output blocks (11 input rows each), default weighted rounding.  Ends with
// a block barrier.
template <int N, int NT, bool kCoherent>
__device__ void load_and_predict(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t plane,
                                 int Hp, int Wp, int x0, int y0, int mvx, int mvy, uint16_t* __restrict__ s_cur,
                                 uint16_t* __restrict__ s_pred, int16_t* __restrict__ s_stage,
                                 int16_t* __restrict__ s_hbuf) {
    constexpr int SW = N + 7;
    constexpr int SP = tqr_stage_stride(N);
    constexpr int NN = N * N;
    constexpr int CCH = N / 8;  // 16-byte chunks per current row
    const int tid = threadIdx.x;
    const int ix = mvx >> 2, iy = mvy >> 2, fx = mvx & 3, fy = mvy & 3;
    const int wx = x0 + ix - 3, wy = y0 + iy - 3;   // window origin
    const int xa = wx - (((wx % 8) + 8) % 8);       // 8-aligned start at or left of wx
    const int off = wx - xa;                        // staged column of window column 0
    const int mch = (off + SW + 7) / 8;             // chunks per window row
    const int ncur = 3 * N * CCH;
    const int ntask = ncur + (ref ? 3 * SW * mch : 0);
    constexpr int kILP = 2;
#pragma unroll 1
    for (int base = tid; base < ntask; base += NT * kILP) {
        uint4 v[kILP];
#pragma unroll
        for (int j = 0; j < kILP; ++j) {
            const int task = base + j * NT;
            if (task < ncur) {
                const int c = task / (N * CCH), rem = task - c * N * CCH, y = rem / CCH, ch = rem - y * CCH;
                v[j] = __ldg(reinterpret_cast<const uint4*>(cur + (size_t)c * plane + (size_t)(y0 + y) * Wp + x0 + 8 * ch));
            } else if (task < ntask) {
                const int t2 = task - ncur;
                const int c = t2 / (SW * mch), rem = t2 - c * SW * mch, r = rem / mch, ch = rem - r * mch;
                const int yy = min(max(wy + r, 0), Hp - 1), xs = xa + 8 * ch;
                const uint16_t* rowp = ref + (size_t)c * plane + (size_t)yy * Wp;
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
            }
        }
#pragma unroll
        for (int j = 0; j < kILP; ++j) {
            const int task = base + j * NT;
            if (task < ncur) {
                const int c = task / (N * CCH), rem = task - c * N * CCH, y = rem / CCH, ch = rem - y * CCH;
                *reinterpret_cast<uint4*>(s_cur + c * NN + y * N + 8 * ch) = v[j];
            } else if (task < ntask) {
                const int t2 = task - ncur;
                const int c = t2 / (SW * mch), rem = t2 - c * SW * mch, r = rem / mch, ch = rem - r * mch;
                *reinterpret_cast<uint4*>(s_stage + (c * SW + r) * SP + 8 * ch) = v[j];
            }
        }
    }
    if (!ref) {
#pragma unroll 1
        for (int idx = tid; idx < 3 * NN; idx += NT) s_pred[idx] = (uint16_t)kFlat;
        __syncthreads();
        return;
    }
    __syncthreads();
    const uint16_t* st = reinterpret_cast<const uint16_t*>(s_stage);
    if (fx != 0) {
        int tap[8];
        luma_taps(fx, tap);
        constexpr int SPR = N / 8;
#pragma unroll 1
        for (int task = tid; task < 3 * SW * SPR; task += NT) {
            const int cr = task / SPR, xs = (task - cr * SPR) * 8;  // cr = c * SW + r
            const uint16_t* srow = st + cr * SP + xs + off;
            int v[15];
#pragma unroll
            for (int i = 0; i < 15; ++i) v[i] = srow[i];
            int o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int acc = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) acc += tap[i] * v[k + i];
                o[k] = acc >> kShift1;
            }
            uint4 pk;
            pk.x = (uint32_t)(uint16_t)o[0] | ((uint32_t)(uint16_t)o[1] << 16);
            pk.y = (uint32_t)(uint16_t)o[2] | ((uint32_t)(uint16_t)o[3] << 16);
            pk.z = (uint32_t)(uint16_t)o[4] | ((uint32_t)(uint16_t)o[5] << 16);
            pk.w = (uint32_t)(uint16_t)o[6] | ((uint32_t)(uint16_t)o[7] << 16);
            *reinterpret_cast<uint4*>(s_hbuf + cr * N + xs) = pk;
        }
        __syncthreads();
    }
    int vtap[8];
    luma_taps(fy == 0 ? 2 : fy, vtap);
    constexpr int B4 = N / 4;
#pragma unroll 1
    for (int task = tid; task < 3 * B4 * B4; task += NT) {
        const int c = task / (B4 * B4), rem = task - c * B4 * B4;
        const int yb = (rem / B4) * 4, xb = (rem - (rem / B4) * B4) * 4;
        int o[4][4];
        if (fy == 0) {
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const int r = yb + y + 3;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    o[y][k] = wp_round(fx ? (int)s_hbuf[(c * SW + r) * N + xb + k]
                                          : (int)st[(c * SW + r) * SP + xb + k + 3 + off] << kShift3);
            }
        } else {
#pragma unroll
            for (int y = 0; y < 4; ++y)
#pragma unroll
                for (int k = 0; k < 4; ++k) o[y][k] = 0;
#pragma unroll
            for (int rho = 0; rho < 11; ++rho) {
                const int r = yb + rho;
                int v[4];
                if (fx) {
                    const uint2 q = *reinterpret_cast<const uint2*>(s_hbuf + (c * SW + r) * N + xb);
                    v[0] = (int)(int16_t)(q.x & 0xffffu); v[1] = (int)q.x >> 16;
                    v[2] = (int)(int16_t)(q.y & 0xffffu); v[3] = (int)q.y >> 16;
                } else {
                    const uint16_t* sr = st + (c * SW + r) * SP + xb + 3 + off;
                    v[0] = sr[0]; v[1] = sr[1]; v[2] = sr[2]; v[3] = sr[3];
                }
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int t = rho - y;
                    if (t >= 0 && t < 8)
#pragma unroll
                        for (int k = 0; k < 4; ++k) o[y][k] += vtap[t] * v[k];
                }
            }
            const int sh = fx ? kShift2 : kShift1;
#pragma unroll
            for (int y = 0; y < 4; ++y)
#pragma unroll
                for (int k = 0; k < 4; ++k) o[y][k] = wp_round(o[y][k] >> sh);
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            uint2 pk;
            pk.x = (uint32_t)o[y][0] | ((uint32_t)o[y][1] << 16);
            pk.y = (uint32_t)o[y][2] | ((uint32_t)o[y][3] << 16);
            *reinterpret_cast<uint2*>(s_pred + c * NN + (yb + y) * N + xb) = pk;
        }
    }
    __syncthreads();
}

// TS consecutive samples of a row (16-byte aligned for TS >= 8, 8-byte for 4).
template <int TS, bool kSigned>
__device__ __forceinline__ void load_seg(const void* p, int (&v)[TS]) {
    if constexpr (TS == 4) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const uint32_t w[2] = {q.x, q.y};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            v[2 * i] = kSigned ? (int)(int16_t)(w[i] & 0xffffu) : (int)(w[i] & 0xffffu);
            v[2 * i + 1] = kSigned ? (int)w[i] >> 16 : (int)(w[i] >> 16);
        }
    } else {
#pragma unroll
        for (int k = 0; k < TS / 8; ++k) {
            const uint4 q = reinterpret_cast<const uint4*>(p)[k];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[8 * k + 2 * i] = kSigned ? (int)(int16_t)(w[i] & 0xffffu) : (int)(w[i] & 0xffffu);
                v[8 * k + 2 * i + 1] = kSigned ? (int)w[i] >> 16 : (int)(w[i] >> 16);
            }
        }
    }
}
template <int TS>
__device__ __forceinline__ void store_seg(void* p, const int (&v)[TS]) {
    if constexpr (TS == 4) {
        uint2 q;
        q.x = (uint32_t)(uint16_t)v[0] | ((uint32_t)(uint16_t)v[1] << 16);
        q.y = (uint32_t)(uint16_t)v[2] | ((uint32_t)(uint16_t)v[3] << 16);
        *reinterpret_cast<uint2*>(p) = q;
    } else {
#pragma unroll
        for (int k = 0; k < TS / 8; ++k) {
            uint4 q;
            q.x = (uint32_t)(uint16_t)v[8 * k] | ((uint32_t)(uint16_t)v[8 * k + 1] << 16);
            q.y = (uint32_t)(uint16_t)v[8 * k + 2] | ((uint32_t)(uint16_t)v[8 * k + 3] << 16);
            q.z = (uint32_t)(uint16_t)v[8 * k + 4] | ((uint32_t)(uint16_t)v[8 * k + 5] << 16);
            q.w = (uint32_t)(uint16_t)v[8 * k + 6] | ((uint32_t)(uint16_t)v[8 * k + 7] << 16);
            reinterpret_cast<uint4*>(p)[k] = q;
        }
    }
}

// One TU size over the whole CU; returns (SSE, bits) through the reduction.
template <int N, int TS, int NT>
__device__ void tu_pass(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ pred,
                        int16_t* __restrict__ work, int16_t* __restrict__ lev, uint16_t* __restrict__ rec,
                        int qp, uint64_t& sse_out, uint32_t& bits_out, uint64_t* red, int slot = -1) {
    constexpr int L = TS == 4 ? 2 : TS == 8 ? 3 : TS == 16 ? 4 : 5;
    constexpr int NTU = N / TS;            // TUs per CU side
    constexpr int TASKS = 3 * N * NTU;     // rows (or columns) of all TUs of all channels
    const int tid = threadIdx.x;
    const QuantParams q = quant_params(qp, L);
    // forward rows
#pragma unroll 1
    for (int t = tid; t < TASKS; t += NT) {
        int c = t / (N * NTU), rem = t - c * N * NTU;
        int y = rem / NTU, tx = rem - y * NTU;
        const int base = c * N * N + y * N + tx * TS;
        int x[TS], yv[TS];
        load_seg<TS, false>(cur + base, x);
        load_seg<TS, false>(pred + base, yv);
#pragma unroll
        for (int i = 0; i < TS; ++i) x[i] -= yv[i];
        fwd1d<TS>(x, yv);
#pragma unroll
        for (int i = 0; i < TS; ++i) yv[i] = rshift_round(yv[i], L + kBitDepth - 9);
        store_seg<TS>(work + base, yv);
    }
    __syncthreads();
    // columns: forward, quantise, dequantise, inverse
    uint32_t bits = 0;
#pragma unroll 1
    for (int t = tid; t < TASKS; t += NT) {
        int c = t / (N * NTU), rem = t - c * N * NTU;
        int ty = rem / N, x = rem - ty * N;
        const int base = c * N * N + ty * TS * N + x;
        int col[TS], cf[TS];
#pragma unroll
        for (int i = 0; i < TS; ++i) col[i] = work[base + i * N];
        fwd1d<TS>(col, cf);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int lv = quant_rate_deq(rshift_round(cf[i], L + 6), q, L, bits, col[i]);
            lev[base + i * N] = (int16_t)lv;
        }
        inv1d<TS>(col, cf);
#pragma unroll
        for (int i = 0; i < TS; ++i) work[base + i * N] = (int16_t)clip16(rshift_round(cf[i], 7));
    }
    __syncthreads();
    // inverse rows and reconstruction; the SSE of a thread fits 32 bits (at
    // most 3 N^2 / NT <= 384 samples of error <= 1023)
    uint32_t sse32 = 0;
#pragma unroll 1
    for (int t = tid; t < TASKS; t += NT) {
        int c = t / (N * NTU), rem = t - c * N * NTU;
        int y = rem / NTU, tx = rem - y * NTU;
        const int base = c * N * N + y * N + tx * TS;
        int e[TS], r[TS];
        load_seg<TS, true>(work + base, e);
        inv1d<TS>(e, r);
        load_seg<TS, false>(pred + base, e);
#pragma unroll
        for (int i = 0; i < TS; ++i) r[i] = clip_pix(e[i] + rshift_round(r[i], 20 - kBitDepth));
        store_seg<TS>(rec + base, r);
        load_seg<TS, false>(cur + base, e);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int d = e[i] - r[i];
            sse32 += (uint32_t)(d * d);
        }
    }
    uint64_t sse = sse32;
    if (slot >= 0) block_sum2_slot<NT>(sse, bits, red, slot);
    else block_sum2<NT>(sse, bits, red);
    sse_out = sse;
    bits_out = bits + 3u * NTU * NTU;  // one coded-block flag per TU and channel
}

// tu_pass for 32 x 32 TUs with two lanes per TU row or column (lane part p
// = the lane's parity, partners in adjacent lanes): each row or column task
// would otherwise leave most of the block idle (3 N tasks per pass), and its
// 32-point transforms are long dependent chains.  The lanes split every
// 32-point transform in halves (fwd32_half / inv32_half, coefficient table
// `tab`); in the column pass each lane quantises its 16 coefficients and the
// two exchange their dequantised halves by shuffle before the inverse.
template <int N, int NT>
__device__ void tu_pass32(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ pred,
                          int16_t* __restrict__ work, int16_t* __restrict__ lev, uint16_t* __restrict__ rec, int qp,
                          const int* __restrict__ tab, uint64_t& sse_out, uint32_t& bits_out, uint64_t* red,
                          int slot = -1) {
    constexpr int L = 5;
    constexpr int NTU = N / 32;
    constexpr int TASKS = 2 * 3 * N * NTU;  // two lanes per TU row (or column) of every channel
    static_assert(NT % 2 == 0, "lane pairs");
    const int tid = threadIdx.x;
    const QuantParams q = quant_params(qp, L);
    const unsigned pmask = 3u << ((threadIdx.x & 31) & ~1u);
    // forward rows: lane part p writes y[16p .. 16p + 15]
#pragma unroll 1
    for (int t = tid; t < TASKS; t += NT) {
        const int p = t & 1, task = t >> 1;
        const int c = task / (N * NTU), rem = task - c * N * NTU;
        const int y = rem / NTU, tx = rem - y * NTU;
        const int base = c * N * N + y * N + tx * 32;
        int x[32];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int cv[8], pv[8];
            load_seg<8, false>(cur + base + 8 * k, cv);
            load_seg<8, false>(pred + base + 8 * k, pv);
#pragma unroll
            for (int i = 0; i < 8; ++i) x[8 * k + i] = cv[i] - pv[i];
        }
        int yh[16];
        fwd32_half(x, p, tab, yh);
#pragma unroll
        for (int i = 0; i < 16; ++i) yh[i] = rshift_round(yh[i], L + kBitDepth - 9);
        store_seg<16>(work + base + 16 * p, yh);
    }
    __syncthreads();
    // columns: forward, quantise and dequantise (16 coefficients per lane),
    // exchange, inverse
    uint32_t bits = 0;
#pragma unroll 1
    for (int t = tid; t < TASKS; t += NT) {
        const int p = t & 1, task = t >> 1;
        const int c = task / (N * NTU), rem = task - c * N * NTU;
        const int ty = rem / N, x = rem - ty * N;
        const int base = c * N * N + ty * 32 * N + x;
        int col[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) col[i] = work[base + i * N];
        int cf[16];
        fwd32_half(col, p, tab, cf);
        int d[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int lv = quant_rate_deq(rshift_round(cf[i], L + 6), q, L, bits, d[i]);
            lev[base + (16 * p + i) * N] = (int16_t)lv;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int o = __shfl_xor_sync(pmask, d[i], 1);
            col[i] = p ? o : d[i];
            col[16 + i] = p ? d[i] : o;
        }
        int lo[8], hi[8];
        inv32_half(col, p, tab, lo, hi);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            work[base + (8 * p + i) * N] = (int16_t)clip16(rshift_round(lo[i], 7));
            work[base + (24 - 8 * p + i) * N] = (int16_t)clip16(rshift_round(hi[i], 7));
        }
    }
    __syncthreads();
    // inverse rows and reconstruction: lane part p rebuilds x[8p .. 8p + 7]
    // and x[24 - 8p .. 31 - 8p]; the SSE of a thread fits 32 bits
    uint32_t sse32 = 0;
#pragma unroll 1
    for (int t = tid; t < TASKS; t += NT) {
        const int p = t & 1, task = t >> 1;
        const int c = task / (N * NTU), rem = task - c * N * NTU;
        const int y = rem / NTU, tx = rem - y * NTU;
        const int base = c * N * N + y * N + tx * 32;
        int e[32];
        load_seg<32, true>(work + base, e);
        int lo[8], hi[8];
        inv32_half(e, p, tab, lo, hi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int off = h == 0 ? 8 * p : 24 - 8 * p;
            int v[8], pr[8], cu[8];
            load_seg<8, false>(pred + base + off, pr);
            load_seg<8, false>(cur + base + off, cu);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                v[i] = clip_pix(pr[i] + rshift_round(h == 0 ? lo[i] : hi[i], 20 - kBitDepth));
                const int dd = cu[i] - v[i];
                sse32 += (uint32_t)(dd * dd);
            }
            store_seg<8>(rec + base + off, v);
        }
    }
    uint64_t sse = sse32;
    if (slot >= 0) block_sum2_slot<NT>(sse, bits, red, slot);
    else block_sum2<NT>(sse, bits, red);
    sse_out = sse;
    bits_out = bits + 3u * NTU * NTU;  // one coded-block flag per TU and channel
}

// Writes the kept reconstruction (and levels) of the CU, 16 bytes per store.
template <int N, int NT>
__device__ __forceinline__ void copy_out(const uint16_t* __restrict__ rec, const int16_t* __restrict__ lev,
                                         uint16_t* __restrict__ recon, int16_t* __restrict__ levels,
                                         int64_t plane, int Wp, int x0, int y0) {
    constexpr int CCH = N / 8;
    for (int t = threadIdx.x; t < 3 * N * CCH; t += NT) {
        const int c = t / (N * CCH), rem = t - c * N * CCH, y = rem / CCH, ch = rem - y * CCH;
        const int si = c * N * N + y * N + 8 * ch;
        const size_t o = (size_t)c * plane + (size_t)(y0 + y) * Wp + x0 + 8 * ch;
        *reinterpret_cast<uint4*>(recon + o) = *reinterpret_cast<const uint4*>(rec + si);
        if (levels) *reinterpret_cast<uint4*>(levels + o) = *reinterpret_cast<const uint4*>(lev + si);
    }
}

// ---------------------------------------------------------------------------
// Low-latency variant for CUs up to 16: all allowed TU sizes are processed at
// once (each has its own work/level/recon buffers), so the whole CU takes
// about seven block barriers instead of three per size.  Same definitions,
// same results.
template <int N>
__host__ __device__ constexpr int tqr_nslots() { return N >= 16 ? 3 : (N >= 8 ? 2 : 1); }
__host__ __device__ constexpr size_t tqr_conc_off_stage(int N) { return align16((size_t)2 * 3 * N * N * 2); }
__host__ __device__ constexpr size_t tqr_conc_off_hbuf(int N) { return tqr_conc_off_stage(N) + tqr_stage_bytes(N); }
__host__ __device__ constexpr size_t tqr_conc_off_slots(int N) { return tqr_conc_off_hbuf(N) + tqr_hbuf_bytes(N); }
__host__ __device__ constexpr size_t tqr_conc_slot_bytes(int N) {
    return align16((size_t)3 * 3 * N * N * 2) + align16((size_t)3 * N * N * 4);
}
__host__ __device__ constexpr size_t tqr_conc_off_acc(int N) { return tqr_conc_off_slots(N) + 3 * tqr_conc_slot_bytes(N); }
__host__ __device__ constexpr size_t tqr_conc_smem_bytes(int N) { return tqr_conc_off_acc(N) + 3 * 8 + 3 * 4 + 16; }

template <int N, int TS>
__device__ __forceinline__ void conc_row_fwd(int lt, const uint16_t* __restrict__ cur, const uint16_t* __restrict__ pred,
                                             int16_t* __restrict__ work) {
    constexpr int L = TS == 4 ? 2 : TS == 8 ? 3 : TS == 16 ? 4 : 5;
    constexpr int NTU = N / TS;
    const int c = lt / (N * NTU), rem = lt - c * N * NTU;
    const int y = rem / NTU, tx = rem - y * NTU;
    const int base = c * N * N + y * N + tx * TS;
    int x[TS], yv[TS];
#pragma unroll
    for (int i = 0; i < TS; ++i) x[i] = (int)cur[base + i] - (int)pred[base + i];
    fwd1d<TS>(x, yv);
#pragma unroll
    for (int i = 0; i < TS; ++i) work[base + i] = (int16_t)rshift_round(yv[i], L + kBitDepth - 9);
}

// Forward column transform of one TU column: coefficients C = rs(T Y, log2N + 6).
template <int N, int TS>
__device__ __forceinline__ void conc_col_fwd(int lt, const int16_t* __restrict__ work, int* __restrict__ coef) {
    constexpr int L = TS == 4 ? 2 : TS == 8 ? 3 : TS == 16 ? 4 : 5;
    constexpr int NTU = N / TS;
    const int c = lt / (N * NTU), rem = lt - c * N * NTU;
    const int ty = rem / N, x = rem - ty * N;
    const int base = c * N * N + ty * TS * N + x;
    int col[TS], cf[TS];
#pragma unroll
    for (int i = 0; i < TS; ++i) col[i] = work[base + i * N];
    fwd1d<TS>(col, cf);
#pragma unroll
    for (int i = 0; i < TS; ++i) coef[base + i * N] = rshift_round(cf[i], L + 6);
}

// Inverse column transform of one TU column of dequantised coefficients:
// E = clip16(rs(T^T D, 7)).
template <int N, int TS>
__device__ __forceinline__ void conc_col_inv(int lt, const int* __restrict__ coef, int16_t* __restrict__ work) {
    constexpr int NTU = N / TS;
    const int c = lt / (N * NTU), rem = lt - c * N * NTU;
    const int ty = rem / N, x = rem - ty * N;
    const int base = c * N * N + ty * TS * N + x;
    int col[TS], r[TS];
#pragma unroll
    for (int i = 0; i < TS; ++i) col[i] = coef[base + i * N];
    inv1d<TS>(col, r);
#pragma unroll
    for (int i = 0; i < TS; ++i) work[base + i * N] = (int16_t)clip16(rshift_round(r[i], 7));
}

template <int N, int TS>
__device__ __forceinline__ uint64_t conc_row_inv(int lt, const uint16_t* __restrict__ cur,
                                                 const uint16_t* __restrict__ pred, const int16_t* __restrict__ work,
                                                 uint16_t* __restrict__ rec) {
    constexpr int NTU = N / TS;
    const int c = lt / (N * NTU), rem = lt - c * N * NTU;
    const int y = rem / NTU, tx = rem - y * NTU;
    const int base = c * N * N + y * N + tx * TS;
    int e[TS], r[TS];
    uint64_t sse = 0;
#pragma unroll
    for (int i = 0; i < TS; ++i) e[i] = work[base + i];
    inv1d<TS>(e, r);
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        int v = clip_pix((int)pred[base + i] + rshift_round(r[i], 20 - kBitDepth));
        rec[base + i] = (uint16_t)v;
        int d = (int)cur[base + i] - v;
        sse += (uint64_t)(d * d);
    }
    return sse;
}

template <int N, int NT, bool kCoherent, bool kPredGiven>
__device__ uint32_t tqr_cu_conc(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t plane,
                                int Hp, int Wp, int x0, int y0, int mvx, int mvy, int qp, unsigned tu_mask,
                                int64_t lf8, uint16_t* __restrict__ recon, int16_t* __restrict__ levels,
                                uint8_t* tu_log2, unsigned char* smem) {
    constexpr int NS = tqr_nslots<N>();
    constexpr int NN = N * N;
    const int tid = threadIdx.x;
    uint16_t* s_cur = reinterpret_cast<uint16_t*>(smem);
    uint16_t* s_pred = s_cur + 3 * NN;
    int16_t* s_stage = reinterpret_cast<int16_t*>(smem + tqr_conc_off_stage(N));
    int16_t* s_hbuf = reinterpret_cast<int16_t*>(smem + tqr_conc_off_hbuf(N));
    unsigned char* slots = smem + tqr_conc_off_slots(N);
    unsigned long long* s_sse = reinterpret_cast<unsigned long long*>(smem + tqr_conc_off_acc(N));
    unsigned* s_bits = reinterpret_cast<unsigned*>(s_sse + 3);
    auto work_of = [&](int s) { return reinterpret_cast<int16_t*>(slots + s * tqr_conc_slot_bytes(N)); };
    auto lev_of = [&](int s) { return work_of(s) + 3 * NN; };
    auto rec_of = [&](int s) { return reinterpret_cast<uint16_t*>(work_of(s) + 6 * NN); };
    auto coef_of = [&](int s) {
        return reinterpret_cast<int*>(slots + s * tqr_conc_slot_bytes(N) + align16((size_t)3 * 3 * NN * 2));
    };

    // 1. current samples, motion-compensated prediction (kPredGiven: the
    // caller has put both in shared memory, s_cur and s_pred)
    if (tid < 3) { s_sse[tid] = 0ull; s_bits[tid] = 0u; }
    if constexpr (kPredGiven) __syncthreads();
    else load_and_predict<N, NT, kCoherent>(cur, ref, plane, Hp, Wp, x0, y0, mvx, mvy, s_cur, s_pred, s_stage, s_hbuf);

    // task ranges of the allowed sizes (slot s: TU size 4 << s)
    int cum[NS + 1];
    cum[0] = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) cum[s + 1] = cum[s] + (((tu_mask >> (s + 2)) & 1u) ? 3 * N * (N / (4 << s)) : 0);
    const int TOT = cum[NS];

    // 2. forward rows, all sizes
#pragma unroll 1
    for (int t = tid; t < TOT; t += NT) {
        int s = 0;
        while (s < NS - 1 && t >= cum[s + 1]) ++s;
        const int lt = t - cum[s];
        if (s == 0) conc_row_fwd<N, 4>(lt, s_cur, s_pred, work_of(0));
        if constexpr (NS > 1) if (s == 1) conc_row_fwd<N, 8>(lt, s_cur, s_pred, work_of(1));
        if constexpr (NS > 2) if (s == 2) conc_row_fwd<N, 16>(lt, s_cur, s_pred, work_of(2));
    }
    __syncthreads();
    // 3. columns: forward transform; then quantise / dequantise element by
    // element over every coefficient of every size (balanced over the block);
    // then the inverse column transform
    uint32_t bitsS[NS];
    uint64_t sseS[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { bitsS[s] = 0; sseS[s] = 0; }
#pragma unroll 1
    for (int t = tid; t < TOT; t += NT) {
        int s = 0;
        while (s < NS - 1 && t >= cum[s + 1]) ++s;
        const int lt = t - cum[s];
        if (s == 0) conc_col_fwd<N, 4>(lt, work_of(0), coef_of(0));
        if constexpr (NS > 1) if (s == 1) conc_col_fwd<N, 8>(lt, work_of(1), coef_of(1));
        if constexpr (NS > 2) if (s == 2) conc_col_fwd<N, 16>(lt, work_of(2), coef_of(2));
    }
    __syncthreads();
    {
        QuantParams qs[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) qs[s] = quant_params(qp, s + 2);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (!((tu_mask >> (s + 2)) & 1u)) continue;
            int* cf = coef_of(s);
            int16_t* lv = lev_of(s);
            for (int i = tid; i < 3 * NN; i += NT) {
                int d;
                lv[i] = (int16_t)quant_rate_deq(cf[i], qs[s], s + 2, bitsS[s], d);
                cf[i] = d;
            }
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int t = tid; t < TOT; t += NT) {
        int s = 0;
        while (s < NS - 1 && t >= cum[s + 1]) ++s;
        const int lt = t - cum[s];
        if (s == 0) conc_col_inv<N, 4>(lt, coef_of(0), work_of(0));
        if constexpr (NS > 1) if (s == 1) conc_col_inv<N, 8>(lt, coef_of(1), work_of(1));
        if constexpr (NS > 2) if (s == 2) conc_col_inv<N, 16>(lt, coef_of(2), work_of(2));
    }
    __syncthreads();
    // 4. inverse rows, reconstruction, SSE
#pragma unroll 1
    for (int t = tid; t < TOT; t += NT) {
        int s = 0;
        while (s < NS - 1 && t >= cum[s + 1]) ++s;
        const int lt = t - cum[s];
        if (s == 0) sseS[0] += conc_row_inv<N, 4>(lt, s_cur, s_pred, work_of(0), rec_of(0));
        if constexpr (NS > 1) if (s == 1) sseS[1] += conc_row_inv<N, 8>(lt, s_cur, s_pred, work_of(1), rec_of(1));
        if constexpr (NS > 2) if (s == 2) sseS[2] += conc_row_inv<N, 16>(lt, s_cur, s_pred, work_of(2), rec_of(2));
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        uint64_t a = sseS[s];
        uint32_t b = bitsS[s];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if ((tid & 31) == 0 && (a | b)) {
            atomicAdd(&s_sse[s], (unsigned long long)a);
            atomicAdd(&s_bits[s], b);
        }
    }
    __syncthreads();
    // 5. the size with the least J (ascending, ties to the larger), copied out
    int64_t bestJ = INT64_MAX;
    int best = 0;
    uint32_t bestBits = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (!((tu_mask >> (s + 2)) & 1u)) continue;
        const int ntu = (N / (4 << s)) * (N / (4 << s));
        const uint32_t bits = s_bits[s] + 3u * ntu;
        const int64_t J = (int64_t)(s_sse[s] << 8) + lf8 * (int64_t)bits;
        if (J <= bestJ) { bestJ = J; best = s; bestBits = bits; }
    }
    copy_out<N, NT>(rec_of(best), lev_of(best), recon, levels, plane, Wp, x0, y0);
    if (tid == 0 && tu_log2) *tu_log2 = (uint8_t)(best + 2);
    uint32_t mvbits = ref ? (uint32_t)(se_len(mvx) + se_len(mvy)) : 0u;
    return 2u + mvbits + bestBits;
}

__host__ __device__ constexpr size_t tqr_smem_bytes(int N) {
    return N <= 16 ? tqr_conc_smem_bytes(N) : tqr_seq_smem_bytes(N);
}

// ---------------------------------------------------------------------------
// CTU 32 with 192 threads (six warps).  Warp w = 2c + h owns rows 16h ..
// 16h + 15 of channel c for every TU size up to 16, so those passes exchange
// data through shared memory within the warp only (__syncwarp): 4 x 4 TUs
// one per lane, entirely in registers; 8 x 8 TUs four lanes each; 16 x 16
// TUs sixteen lanes each.  The 32 x 32 TU of a channel pairs the channel's
// two warps (a 64-thread named barrier between its passes).  Each size
// writes its levels and reconstruction into whichever of two buffers does
// not hold the best size so far; one block barrier per size makes its
// totals known, and the best buffer is copied out once at the end.  Same
// definitions and results as tqr_cu_seq.
//
// Shared memory: cur, pred, work ([3][32][32] each), buffers 0 and 1 (levels
// int16 then reconstruction u16, [3][32][32] each), the per-size sums, the
// 32-point table.  The motion-compensation staging and its horizontal pass
// live in the two buffers until the prediction is done.
constexpr int kW32Threads = 192;
__host__ __device__ constexpr size_t w32_plane_bytes() { return (size_t)3 * 32 * 32 * 2; }
__host__ __device__ constexpr size_t w32_off_buf(int i) { return (3 + 2 * (size_t)i) * w32_plane_bytes(); }
__host__ __device__ constexpr size_t w32_off_red() { return w32_off_buf(2); }
__host__ __device__ constexpr size_t w32_off_t32() { return w32_off_red() + 8 * 8; }
__host__ __device__ constexpr size_t tqr_w32_smem_bytes() { return w32_off_t32() + (size_t)kT32HalvesInts * 4; }
static_assert(tqr_stage_bytes(32) + tqr_hbuf_bytes(32) <= 4 * w32_plane_bytes(), "staging fits the two buffers");
static_assert(tqr_w32_smem_bytes() <= tqr_seq_smem_bytes(32), "fits every caller's CTU-32 allocation");

// Warp sums of (sse, bits) added to slot `slot` (sse at red[slot], bits at
// red[4 + slot]).  A warp's SSE fits 32 bits: 512 samples of error <= 1023.
__device__ __forceinline__ void w32_warp_sums(uint32_t sse, uint32_t bits, unsigned long long* red, int slot) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sse += __shfl_xor_sync(0xffffffffu, sse, o);
        bits += __shfl_xor_sync(0xffffffffu, bits, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red + slot, (unsigned long long)sse);
        atomicAdd(red + 4 + slot, (unsigned long long)bits);
    }
}

// 4 x 4 TUs: lane = (TU row 0..3, TU column 0..7) of the warp's region.
__device__ __forceinline__ void w32_tu4(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ pred,
                                        int16_t* __restrict__ lev, uint16_t* __restrict__ rec, const QuantParams& q,
                                        int rbase, int lane, uint32_t& sse, uint32_t& bits) {
    constexpr int L = 2;
    const int base = rbase + (lane >> 3) * 4 * 32 + (lane & 7) * 4;
    int x[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int cv[4], pv[4];
        load_seg<4, false>(cur + base + 32 * i, cv);
        load_seg<4, false>(pred + base + 32 * i, pv);
        int y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cv[k] -= pv[k];
        fwd1d<4>(cv, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) x[i][k] = rshift_round(y[k], L + kBitDepth - 9);
    }
    int lv[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int col[4], cf[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) col[i] = x[i][k];
        fwd1d<4>(col, cf);
#pragma unroll
        for (int i = 0; i < 4; ++i) lv[i][k] = quant_rate_deq(rshift_round(cf[i], L + 6), q, L, bits, col[i]);
        inv1d<4>(col, cf);
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i][k] = clip16(rshift_round(cf[i], 7));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        store_seg<4>(lev + base + 32 * i, lv[i]);
        int r[4], cv[4], pv[4];
        inv1d<4>(x[i], r);
        load_seg<4, false>(pred + base + 32 * i, pv);
        load_seg<4, false>(cur + base + 32 * i, cv);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            r[k] = clip_pix(pv[k] + rshift_round(r[k], 20 - kBitDepth));
            const int d = cv[k] - r[k];
            sse += (uint32_t)(d * d);
        }
        store_seg<4>(rec + base + 32 * i, r);
    }
}

// 8 x 8 and 16 x 16 TUs over the warp's region (16 rows x 32 columns, row
// stride 32): rows forward (task = row and TU column), columns forward,
// quantised, dequantised and inverted (task = column and TU row), rows
// inverse with the reconstruction; the work plane between the passes.
template <int TS>
__device__ __forceinline__ void w32_tu(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ pred,
                                       int16_t* __restrict__ work, int16_t* __restrict__ lev,
                                       uint16_t* __restrict__ rec, const QuantParams& q, int rbase, int lane,
                                       uint32_t& sse, uint32_t& bits) {
    constexpr int L = TS == 8 ? 3 : 4;
    constexpr int NTU = 32 / TS;        // TU columns in the region
    constexpr int R = 16 * NTU / 32;    // row tasks per lane (16 rows x NTU TU columns)
    constexpr int C = 32 * (16 / TS) / 32;  // column tasks per lane (32 columns x 16/TS TU rows)
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
        const int t = lane + 32 * j;
        const int o = rbase + (t / NTU) * 32 + (t % NTU) * TS;
        int x[TS], yv[TS];
        load_seg<TS, false>(cur + o, x);
        load_seg<TS, false>(pred + o, yv);
#pragma unroll
        for (int i = 0; i < TS; ++i) x[i] -= yv[i];
        fwd1d<TS>(x, yv);
#pragma unroll
        for (int i = 0; i < TS; ++i) yv[i] = rshift_round(yv[i], L + kBitDepth - 9);
        store_seg<TS>(work + o, yv);
    }
    __syncwarp();
#pragma unroll 1
    for (int j = 0; j < C; ++j) {
        const int o = rbase + j * TS * 32 + lane;
        int col[TS], cf[TS];
#pragma unroll
        for (int i = 0; i < TS; ++i) col[i] = work[o + 32 * i];
        fwd1d<TS>(col, cf);
#pragma unroll
        for (int i = 0; i < TS; ++i)
            lev[o + 32 * i] = (int16_t)quant_rate_deq(rshift_round(cf[i], L + 6), q, L, bits, col[i]);
        inv1d<TS>(col, cf);
#pragma unroll
        for (int i = 0; i < TS; ++i) work[o + 32 * i] = (int16_t)clip16(rshift_round(cf[i], 7));
    }
    __syncwarp();
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
        const int t = lane + 32 * j;
        const int o = rbase + (t / NTU) * 32 + (t % NTU) * TS;
        int e[TS], r[TS];
        load_seg<TS, true>(work + o, e);
        inv1d<TS>(e, r);
        load_seg<TS, false>(pred + o, e);
#pragma unroll
        for (int i = 0; i < TS; ++i) r[i] = clip_pix(e[i] + rshift_round(r[i], 20 - kBitDepth));
        store_seg<TS>(rec + o, r);
        load_seg<TS, false>(cur + o, e);
#pragma unroll
        for (int i = 0; i < TS; ++i) {
            const int d = e[i] - r[i];
            sse += (uint32_t)(d * d);
        }
    }
}

// 64-thread barrier of channel c's two warps (named barriers 1 .. 3).
__device__ __forceinline__ void w32_pair_sync(int c) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + c) : "memory");
}

// The 32 x 32 TU of channel c by its two warps, two lanes per row or column
// (t = 32 h + lane; lane part p = t & 1), as in tu_pass32.
__device__ __forceinline__ void w32_tu32(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ pred,
                                         int16_t* __restrict__ work, int16_t* __restrict__ lev,
                                         uint16_t* __restrict__ rec, const QuantParams& q,
                                         const int* __restrict__ tab, int c, int t, uint32_t& sse, uint32_t& bits) {
    constexpr int L = 5;
    const int p = t & 1, v = t >> 1;
    const int cb = c * 1024;
    const unsigned pmask = 3u << ((threadIdx.x & 31) & ~1u);
    {  // forward row v: lane part p writes y[16p .. 16p + 15]
        const int base = cb + v * 32;
        int x[32];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int cv[8], pv[8];
            load_seg<8, false>(cur + base + 8 * k, cv);
            load_seg<8, false>(pred + base + 8 * k, pv);
#pragma unroll
            for (int i = 0; i < 8; ++i) x[8 * k + i] = cv[i] - pv[i];
        }
        int yh[16];
        fwd32_half(x, p, tab, yh);
#pragma unroll
        for (int i = 0; i < 16; ++i) yh[i] = rshift_round(yh[i], L + kBitDepth - 9);
        store_seg<16>(work + base + 16 * p, yh);
    }
    w32_pair_sync(c);
    {  // column v: forward, quantise, dequantise (16 coefficients per lane), exchange, inverse
        const int base = cb + v;
        int col[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) col[i] = work[base + i * 32];
        int cf[16];
        fwd32_half(col, p, tab, cf);
        int d[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            lev[base + (16 * p + i) * 32] = (int16_t)quant_rate_deq(rshift_round(cf[i], L + 6), q, L, bits, d[i]);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int o = __shfl_xor_sync(pmask, d[i], 1);
            col[i] = p ? o : d[i];
            col[16 + i] = p ? d[i] : o;
        }
        int lo[8], hi[8];
        inv32_half(col, p, tab, lo, hi);
        // every lane of the pair has read the whole column before either writes it
        __syncwarp(pmask);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            work[base + (8 * p + i) * 32] = (int16_t)clip16(rshift_round(lo[i], 7));
            work[base + (24 - 8 * p + i) * 32] = (int16_t)clip16(rshift_round(hi[i], 7));
        }
    }
    w32_pair_sync(c);
    {  // inverse row v and reconstruction: lane part p rebuilds x[8p .. 8p + 7] and x[24 - 8p .. 31 - 8p]
        const int base = cb + v * 32;
        int e[32];
        load_seg<32, true>(work + base, e);
        int lo[8], hi[8];
        inv32_half(e, p, tab, lo, hi);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int off = hh == 0 ? 8 * p : 24 - 8 * p;
            int vv[8], pr[8], cu[8];
            load_seg<8, false>(pred + base + off, pr);
            load_seg<8, false>(cur + base + off, cu);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                vv[i] = clip_pix(pr[i] + rshift_round(hh == 0 ? lo[i] : hi[i], 20 - kBitDepth));
                const int dd = cu[i] - vv[i];
                sse += (uint32_t)(dd * dd);
            }
            store_seg<8>(rec + base + off, vv);
        }
    }
}

template <bool kCoherent>
__device__ uint32_t tqr_cu_w32(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t plane,
                               int Hp, int Wp, int x0, int y0, int mvx, int mvy, int qp, unsigned tu_mask,
                               int64_t lf8, uint16_t* __restrict__ recon, int16_t* __restrict__ levels,
                               uint8_t* tu_log2, unsigned char* smem) {
    constexpr int N = 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, c = w >> 1, h = w & 1;
    uint16_t* s_cur = reinterpret_cast<uint16_t*>(smem);
    uint16_t* s_pred = s_cur + 3 * N * N;
    int16_t* s_work = reinterpret_cast<int16_t*>(s_pred + 3 * N * N);
    unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + w32_off_red());
    int* t32tab = reinterpret_cast<int*>(smem + w32_off_t32());
    auto lev_of = [&](int b) { return reinterpret_cast<int16_t*>(smem + w32_off_buf(b)); };
    auto rec_of = [&](int b) { return reinterpret_cast<uint16_t*>(smem + w32_off_buf(b) + w32_plane_bytes()); };

    t32_halves_init(t32tab);  // in flight during the prediction
    if (tid < 8) red[tid] = 0ull;  // the per-size sums (visible after the next barrier)
    load_and_predict<N, kW32Threads, kCoherent>(cur, ref, plane, Hp, Wp, x0, y0, mvx, mvy, s_cur, s_pred,
                                                reinterpret_cast<int16_t*>(smem + w32_off_buf(0)),
                                                reinterpret_cast<int16_t*>(smem + w32_off_buf(0) +
                                                                           tqr_stage_bytes(N)));
    t32_halves_wait();
    __syncthreads();

    const int rbase = c * N * N + 16 * h * N;  // the warp's region
    int64_t bestJ = INT64_MAX;
    int bestL = 0, best = 0, wb = 0;  // best buffer, buffer being written
    uint32_t bestBits = 0;
    // after a size's pass: its totals, and the buffers swapped when it is the best so far
    auto finish = [&](int L, int slot, uint32_t sse, uint32_t bits) {
        w32_warp_sums(sse, bits, red, slot);
        __syncthreads();
        const uint32_t b = (uint32_t)red[4 + slot] + 3u * (uint32_t)((N >> L) * (N >> L));  // + coded-block flags
        const int64_t J = (int64_t)(red[slot] << 8) + lf8 * (int64_t)b;
        if (J <= bestJ) {  // ascending sizes: ties go to the larger
            bestJ = J;
            bestL = L;
            bestBits = b;
            best = wb;
            wb ^= 1;
        }
    };
    if (tu_mask & (1u << 2)) {
        uint32_t sse = 0, bits = 0;
        const QuantParams q = quant_params(qp, 2);
        w32_tu4(s_cur, s_pred, lev_of(wb), rec_of(wb), q, rbase, lane, sse, bits);
        finish(2, 0, sse, bits);
    }
    if (tu_mask & (1u << 3)) {
        uint32_t sse = 0, bits = 0;
        const QuantParams q = quant_params(qp, 3);
        w32_tu<8>(s_cur, s_pred, s_work, lev_of(wb), rec_of(wb), q, rbase, lane, sse, bits);
        finish(3, 1, sse, bits);
    }
    if (tu_mask & (1u << 4)) {
        uint32_t sse = 0, bits = 0;
        const QuantParams q = quant_params(qp, 4);
        w32_tu<16>(s_cur, s_pred, s_work, lev_of(wb), rec_of(wb), q, rbase, lane, sse, bits);
        finish(4, 2, sse, bits);
    }
    if (tu_mask & (1u << 5)) {
        uint32_t sse = 0, bits = 0;
        const QuantParams q = quant_params(qp, 5);
        w32_tu32(s_cur, s_pred, s_work, lev_of(wb), rec_of(wb), q, t32tab, c, 32 * h + lane, sse, bits);
        finish(5, 3, sse, bits);
    }
    copy_out<N, kW32Threads>(rec_of(best), lev_of(best), recon, levels, plane, Wp, x0, y0);
    if (tid == 0 && tu_log2) *tu_log2 = (uint8_t)bestL;
    const uint32_t mvbits = ref ? (uint32_t)(se_len(mvx) + se_len(mvy)) : 0u;
    return 2u + mvbits + bestBits;
}

// Transform/quantise/reconstruct the CU at (x0, y0).  cur/ref/recon/levels:
// the group's frame [3][Hp][Wp] (ref == nullptr: first frame).  Returns the
// CU's rate-proxy bits; writes recon (and levels) and *tu_log2.  kPredGiven:
// the current samples and the prediction are already in shared memory (cur
// u16 [3][N][N] at offset 0, the prediction right after it), written before
// a barrier; cur, ref and the vector are then not read, and the bits count
// no vector (ref must be nullptr).
template <int N, int NT, bool kCoherent, bool kPredGiven>
__device__ uint32_t tqr_cu_seq(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t plane,
                               int Hp, int Wp, int x0, int y0, int mvx, int mvy, int qp, unsigned tu_mask,
                               int64_t lf8, uint16_t* __restrict__ recon, int16_t* __restrict__ levels,
                               uint8_t* tu_log2, unsigned char* smem);

template <int N, int NT, bool kCoherent = false, bool kPredGiven = false>
__device__ uint32_t tqr_cu(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t plane,
                           int Hp, int Wp, int x0, int y0, int mvx, int mvy, int qp, unsigned tu_mask,
                           int64_t lf8, uint16_t* __restrict__ recon, int16_t* __restrict__ levels,
                           uint8_t* tu_log2, unsigned char* smem) {
    if constexpr (N <= 16) {
        return tqr_cu_conc<N, NT, kCoherent, kPredGiven>(cur, ref, plane, Hp, Wp, x0, y0, mvx, mvy, qp, tu_mask,
                                                         lf8, recon, levels, tu_log2, smem);
    } else if constexpr (N == 32 && NT == kW32Threads && !kPredGiven) {
        return tqr_cu_w32<kCoherent>(cur, ref, plane, Hp, Wp, x0, y0, mvx, mvy, qp, tu_mask, lf8, recon, levels,
                                     tu_log2, smem);
    } else {
        return tqr_cu_seq<N, NT, kCoherent, kPredGiven>(cur, ref, plane, Hp, Wp, x0, y0, mvx, mvy, qp, tu_mask, lf8,
                                                        recon, levels, tu_log2, smem);
    }
}

// The size-by-size form: one TU size after another over the whole CU, the
// reconstruction and levels of the best so far copied out as soon as a size
// improves on it.
template <int N, int NT, bool kCoherent, bool kPredGiven>
__device__ uint32_t tqr_cu_seq(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t plane,
                               int Hp, int Wp, int x0, int y0, int mvx, int mvy, int qp, unsigned tu_mask,
                               int64_t lf8, uint16_t* __restrict__ recon, int16_t* __restrict__ levels,
                               uint8_t* tu_log2, unsigned char* smem) {
    const int tid = threadIdx.x;
    uint16_t* s_cur = reinterpret_cast<uint16_t*>(smem);
    uint16_t* s_pred = s_cur + 3 * N * N;
    int16_t* s_work = reinterpret_cast<int16_t*>(s_pred + 3 * N * N);
    int16_t* s_lev = s_work + 3 * N * N;
    uint16_t* s_rec = reinterpret_cast<uint16_t*>(s_lev + 3 * N * N);
    int16_t* s_stage = reinterpret_cast<int16_t*>(smem + tqr_off_stage(N));
    int16_t* s_hbuf = reinterpret_cast<int16_t*>(smem + tqr_off_hbuf(N));
    uint64_t* red = reinterpret_cast<uint64_t*>(smem + tqr_off_red(N));

    int* t32tab = reinterpret_cast<int*>(smem + tqr_off_t32(N));
    if constexpr (N >= 32) t32_halves_init(t32tab);  // in flight during the prediction
    if (tid < 8) red[tid] = 0ull;  // the per-size sum slots (visible after the next barrier)
    if constexpr (!kPredGiven)
        load_and_predict<N, NT, kCoherent>(cur, ref, plane, Hp, Wp, x0, y0, mvx, mvy, s_cur, s_pred, s_stage, s_hbuf);
    if constexpr (N >= 32) {
        t32_halves_wait();
        __syncthreads();
    }

    int64_t bestJ = INT64_MAX;
    int bestL = 0;
    uint32_t bestBits = 0;
    auto consider = [&](int L, uint64_t sse, uint32_t bits) {
        int64_t J = (int64_t)(sse << 8) + lf8 * (int64_t)bits;
        if (J <= bestJ) {  // ascending sizes: ties go to the larger
            bestJ = J;
            bestL = L;
            bestBits = bits;
            copy_out<N, NT>(s_rec, s_lev, recon, levels, plane, Wp, x0, y0);
        }
        // no barrier: the next size's first pass writes only the work planes,
        // and its levels and reconstruction only after its own barriers
    };
    uint64_t sse;
    uint32_t bits;
    if (tu_mask & (1u << 2)) { tu_pass<N, 4, NT>(s_cur, s_pred, s_work, s_lev, s_rec, qp, sse, bits, red, 0); consider(2, sse, bits); }
    if constexpr (N >= 8)
        if (tu_mask & (1u << 3)) { tu_pass<N, 8, NT>(s_cur, s_pred, s_work, s_lev, s_rec, qp, sse, bits, red, 1); consider(3, sse, bits); }
    if constexpr (N >= 16)
        if (tu_mask & (1u << 4)) { tu_pass<N, 16, NT>(s_cur, s_pred, s_work, s_lev, s_rec, qp, sse, bits, red, 2); consider(4, sse, bits); }
    if constexpr (N >= 32)
        if (tu_mask & (1u << 5)) { tu_pass32<N, NT>(s_cur, s_pred, s_work, s_lev, s_rec, qp, t32tab, sse, bits, red, 3); consider(5, sse, bits); }
    if (tid == 0 && tu_log2) *tu_log2 = (uint8_t)bestL;
    uint32_t mvbits = ref ? (uint32_t)(se_len(mvx) + se_len(mvy)) : 0u;
    return 2u + mvbits + bestBits;
}

}  // namespace xvd
