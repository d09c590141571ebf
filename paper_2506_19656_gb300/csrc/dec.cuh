// dec.cuh -- decode one CU by one thread block (device code).
//
// The inverse of tqr_cu for the TU size the encoder kept: the prediction is
// the encoder's (flat 2^(B-1) in frame 0, else the CU's quarter-sample
// vector applied to all three channels of the previous reconstruction), the
// residual is the inverse transform of the dequantised levels
//   columns: E = clip16(rs(T^T D, 7)),  rows: r = rs(E T, 20 - B),
// and recon = clip(pred + r, 0, 1023).  The rate proxy is recomputed from
// the levels: 2 (TU size) + |se(mvx)| + |se(mvy)| (not in frame 0) + per TU
// and channel 1 + sum over nonzero levels of (2 log2N + |se(level)|) -- the
// encoder's count, so a decoder that reproduces it has read the same data.
//
// Shared memory (the sequential transform layout, tqr_seq_smem_bytes):
//   lev int16 [3][N][N] (loaded like the encoder's current samples),
//   pred u16 [3][N][N] (overwritten by the reconstruction), work int16
//   [3][N][N], stage/hbuf (motion compensation; the stage region then holds
//   the dequantised coefficients, int32 [3][N][N]), one bits counter.
#pragma once
#include <cstdint>
#include "tqr.cuh"

namespace xvd {

__host__ __device__ constexpr size_t dec_smem_bytes(int N) { return tqr_seq_smem_bytes(N); }
// the int32 coefficients fit in the stage and hbuf regions, before the reductions
static_assert(12 * 8 * 8 <= tqr_off_red(8) - tqr_off_stage(8) && 12 * 16 * 16 <= tqr_off_red(16) - tqr_off_stage(16) &&
                  12 * 32 * 32 <= tqr_off_red(32) - tqr_off_stage(32) && 12 * 64 * 64 <= tqr_off_red(64) - tqr_off_stage(64),
              "dequantised coefficients overflow the motion-compensation regions");

// Inverse rows of one TU row and the reconstruction, in place over pred.
template <int N, int TS>
__device__ __forceinline__ void dec_row_inv(int lt, const int16_t* __restrict__ work, uint16_t* __restrict__ pred_rec) {
    constexpr int NTU = N / TS;
    const int c = lt / (N * NTU), rem = lt - c * N * NTU;
    const int y = rem / NTU, tx = rem - y * NTU;
    const int base = c * N * N + y * N + tx * TS;
    int e[TS], r[TS];
#pragma unroll
    for (int i = 0; i < TS; ++i) e[i] = work[base + i];
    inv1d<TS>(e, r);
#pragma unroll
    for (int i = 0; i < TS; ++i)
        pred_rec[base + i] = (uint16_t)clip_pix((int)pred_rec[base + i] + rshift_round(r[i], 20 - kBitDepth));
}

// Residual of every TU of size TS over the CU's three channels; returns this
// thread's share of the level bits.
template <int N, int TS, int NT>
__device__ uint32_t dec_tus(const int16_t* __restrict__ s_lev, uint16_t* __restrict__ s_pred, int16_t* __restrict__ s_work,
                            int* __restrict__ s_coef, int qp) {
    constexpr int L = TS == 4 ? 2 : TS == 8 ? 3 : TS == 16 ? 4 : 5;
    constexpr int TASKS = 3 * N * (N / TS);  // TU columns (or rows) of all channels
    const int tid = threadIdx.x;
    const QuantParams q = quant_params(qp, L);
    uint32_t bits = 0;
    for (int i = tid; i < 3 * N * N; i += NT) {
        const int l = s_lev[i];
        if (l != 0) {
            bits += (uint32_t)(2 * L + se_len(l));
            s_coef[i] = dequantize(l, q);
        } else {
            s_coef[i] = 0;
        }
    }
    __syncthreads();
    for (int t = tid; t < TASKS; t += NT) conc_col_inv<N, TS>(t, s_coef, s_work);
    __syncthreads();
    for (int t = tid; t < TASKS; t += NT) dec_row_inv<N, TS>(t, s_work, s_pred);
    __syncthreads();
    return bits;
}

// Decodes the CU at (x0, y0): levels/ref/recon are the group's frame
// [3][Hp][Wp] (ref == nullptr: frame 0); L = the CU's log2 TU size (values
// outside 2..log2 N are clamped into it).  Writes recon; returns the CU's
// rate-proxy bits (the same value on every thread).  kPredGiven: the caller
// has put the CU's levels (int16 [3][N][N] at offset 0) and its prediction
// (right after them) in shared memory before a barrier; levels, ref and the
// vector are then not read, and the bits count no vector.
template <int N, int NT, bool kCoherent = false, bool kPredGiven = false>
__device__ uint32_t dec_cu(const int16_t* __restrict__ levels, const uint16_t* __restrict__ ref, int64_t plane,
                           int Hp, int Wp, int x0, int y0, int mvx, int mvy, int L, int qp,
                           uint16_t* __restrict__ recon, unsigned char* smem) {
    constexpr int NN = N * N;
    constexpr int LN = N == 8 ? 3 : N == 16 ? 4 : N == 32 ? 5 : 6;
    const int tid = threadIdx.x;
    int16_t* s_lev = reinterpret_cast<int16_t*>(smem);
    uint16_t* s_pred = reinterpret_cast<uint16_t*>(s_lev + 3 * NN);
    int16_t* s_work = reinterpret_cast<int16_t*>(s_pred + 3 * NN);
    int16_t* s_stage = reinterpret_cast<int16_t*>(smem + tqr_off_stage(N));
    int16_t* s_hbuf = reinterpret_cast<int16_t*>(smem + tqr_off_hbuf(N));
    int* s_coef = reinterpret_cast<int*>(s_stage);  // after the prediction
    unsigned* s_bits = reinterpret_cast<unsigned*>(smem + tqr_off_red(N));
    if (tid == 0) *s_bits = 0u;
    // the levels have the current samples' layout: one load batch with the
    // motion-compensation windows
    if constexpr (kPredGiven) __syncthreads();
    else
        load_and_predict<N, NT, kCoherent>(reinterpret_cast<const uint16_t*>(levels), ref, plane, Hp, Wp, x0, y0,
                                           mvx, mvy, reinterpret_cast<uint16_t*>(s_lev), s_pred, s_stage, s_hbuf);
    L = L < 2 ? 2 : (L > LN ? LN : L);
    if (L > 5) L = 5;  // no 64-point transform
    uint32_t bits = 0;
    if (L == 2) bits = dec_tus<N, 4, NT>(s_lev, s_pred, s_work, s_coef, qp);
    if constexpr (N >= 8) if (L == 3) bits = dec_tus<N, 8, NT>(s_lev, s_pred, s_work, s_coef, qp);
    if constexpr (N >= 16) if (L == 4) bits = dec_tus<N, 16, NT>(s_lev, s_pred, s_work, s_coef, qp);
    if constexpr (N >= 32) if (L == 5) bits = dec_tus<N, 32, NT>(s_lev, s_pred, s_work, s_coef, qp);
#pragma unroll
    for (int o = 16; o; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
    if ((tid & 31) == 0 && bits) atomicAdd(s_bits, bits);
    __syncthreads();
    copy_out<N, NT>(s_pred, nullptr, recon, nullptr, plane, Wp, x0, y0);
    const int ntu = (N >> L) * (N >> L);
    const uint32_t mvbits = ref ? (uint32_t)(se_len(mvx) + se_len(mvy)) : 0u;
    return 2u + mvbits + 3u * (uint32_t)ntu + *s_bits;
}

}  // namespace xvd
