// xv_dev.cuh -- device-side building blocks of the encoder analysis.
//
// Everything here is integer arithmetic that must match the definitions in
// include/xv.h bit for bit:
//   * the HEVC core-transform matrix (H.265 subclause 8.6.4.2: a 32x32 table
//     of scaled cosines; an N-point transform uses rows k * 32/N), applied by
//     partial butterflies -- an exact re-association of the matrix product;
//   * the HEVC 8-tap luma interpolation filter (H.265 8.5.3.3.3.1);
//   * signed Exp-Golomb code lengths for the motion and level rate proxy.
#pragma once
#include <cstdint>

namespace xvd {

constexpr int kBitDepth = 10;
constexpr int kPixMax = (1 << kBitDepth) - 1;
constexpr int kFlat = 1 << (kBitDepth - 1);  // first-frame prediction value

// ---------------------------------------------------------------- transform
// Scaled cosine 64*sqrt(2)*cos(m*pi/64) as HEVC rounds it, for m = 0..32
// (m = 0 only ever appears in the DC row, whose value is 64).
__host__ __device__ constexpr int hevc_cos(int m) {
    constexpr int c[33] = {64, 90, 90, 90, 89, 88, 87, 85, 83, 82, 80, 78, 75, 73, 70, 67, 64,
                           61, 57, 54, 50, 46, 43, 38, 36, 31, 25, 22, 18, 13, 9,  4,  0};
    return c[m];
}

// Entry (k, n) of the 32-point matrix: DC row 64; otherwise the cosine of
// angle k(2n+1) pi/64, folded into [0, pi/2] with its sign.
__host__ __device__ constexpr int t32(int k, int n) {
    if (k == 0) return 64;
    int a = (k * (2 * n + 1)) & 127;  // angle in units of pi/64, modulo 2 pi
    if (a > 64) a = 128 - a;          // cos(2pi - t) = cos(t)
    return a <= 32 ? hevc_cos(a) : -hevc_cos(64 - a);  // cos(pi - t) = -cos(t)
}

// Entry (k, n) of the N-point matrix: row k * 32/N of the 32-point matrix.
template <int N>
__host__ __device__ constexpr int tN(int k, int n) { return t32(k * (32 / N), n); }

// y[k] = sum_n T_N[k][n] x[n]  (no rounding), partial butterfly.
template <int N>
__device__ __forceinline__ void fwd1d(const int (&x)[N], int (&y)[N]) {
    if constexpr (N == 2) {
        y[0] = 64 * (x[0] + x[1]);
        y[1] = 64 * (x[0] - x[1]);
    } else {
        int e[N / 2], o[N / 2], ye[N / 2];
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            e[k] = x[k] + x[N - 1 - k];
            o[k] = x[k] - x[N - 1 - k];
        }
        fwd1d<N / 2>(e, ye);
#pragma unroll
        for (int i = 0; i < N / 2; ++i) y[2 * i] = ye[i];
#pragma unroll
        for (int k = 1; k < N; k += 2) {
            int acc = 0;
#pragma unroll
            for (int n = 0; n < N / 2; ++n) acc += tN<N>(k, n) * o[n];
            y[k] = acc;
        }
    }
}

// x[n] = sum_k T_N[k][n] c[k]  (no rounding), partial butterfly.
template <int N>
__device__ __forceinline__ void inv1d(const int (&c)[N], int (&x)[N]) {
    if constexpr (N == 2) {
        x[0] = 64 * (c[0] + c[1]);
        x[1] = 64 * (c[0] - c[1]);
    } else {
        int ce[N / 2], ee[N / 2];
#pragma unroll
        for (int i = 0; i < N / 2; ++i) ce[i] = c[2 * i];
        inv1d<N / 2>(ce, ee);
#pragma unroll
        for (int n = 0; n < N / 2; ++n) {
            int o = 0;
#pragma unroll
            for (int i = 0; i < N / 2; ++i) o += tN<N>(2 * i + 1, n) * c[2 * i + 1];
            x[n] = ee[n] + o;
            x[N - 1 - n] = ee[n] - o;
        }
    }
}

__device__ __forceinline__ int rshift_round(int v, int s) { return (v + (1 << (s - 1))) >> s; }

// The 32-point transform shared by two lanes (l and l ^ 1, lane part p = 0
// or 1), both executing the same instructions on different coefficients:
// the even half (a 16-point transform) is computed by both, the 16 x 16 odd
// part is split in two 8 x 16 halves whose coefficients come from a table in
// shared memory (t32_halves_init) instead of instruction immediates.
//   table[0 .. 255]:   forward, [p][j][n] = T32[2 (8p + j) + 1][n]
//   table[256 .. 511]: inverse, [p][i][j] = T32[2j + 1][8p + i]
constexpr int kT32HalvesInts = 512;
// A 16-byte shared-memory load the compiler keeps where it is written: the
// coefficient loads do not depend on the task, and hoisted out of a task
// loop 256 of them would stay in registers.
__device__ __forceinline__ int4 lds_coef4(const int* p) {
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}
struct T32Halves {
    int v[kT32HalvesInts];
};
__host__ __device__ constexpr T32Halves make_t32_halves() {
    T32Halves t{};
    for (int idx = 0; idx < kT32HalvesInts; ++idx) {
        const int inv = idx >> 8, p = (idx >> 7) & 1, a = (idx >> 4) & 7, b = idx & 15;
        t.v[idx] = inv ? t32(2 * b + 1, 8 * p + a) : t32(2 * (8 * p + a) + 1, b);
    }
    return t;
}
// the table, computed at compile time (global memory, read once per CU)
__device__ const T32Halves kT32HalvesTab = make_t32_halves();
// Starts copying the table into shared memory `tab` (16-byte aligned) with
// asynchronous copies, so that no thread waits on the loads here; the
// copying threads must call t32_halves_wait() before a barrier that
// precedes the first use.
__device__ __forceinline__ void t32_halves_init(int* tab) {
    for (int i = threadIdx.x; i < kT32HalvesInts / 4; i += blockDim.x) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(tab + 4 * i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(kT32HalvesTab.v + 4 * i) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void t32_halves_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// y[16p .. 16p + 15] of y = T32 x (x: all 32 samples, on both lanes).  The
// odd part first, so that its inputs are dead before the even part starts.
__device__ __forceinline__ void fwd32_half(const int (&x)[32], int p, const int* __restrict__ tab, int (&y)[16]) {
    int e[16], o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        e[k] = x[k] + x[31 - k];
        o[k] = x[k] - x[31 - k];
    }
    const int* f = tab + p * 128;
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // y[2 (8p + j) + 1] = y[16p + 2j + 1]
        int acc = 0;
#pragma unroll
        for (int n = 0; n < 16; n += 4) {
            const int4 c = lds_coef4(f + j * 16 + n);
            acc += c.x * o[n] + c.y * o[n + 1] + c.z * o[n + 2] + c.w * o[n + 3];
        }
        y[2 * j + 1] = acc;
    }
    int ye[16];
    fwd1d<16>(e, ye);  // y[2i] = ye[i]
#pragma unroll
    for (int j = 0; j < 8; ++j) y[2 * j] = p ? ye[8 + j] : ye[j];
}

// Part of x = T32^T c (c: all 32 coefficients, on both lanes): lo[i] =
// x[8p + i] and hi[i] = x[24 - 8p + i], i < 8.  The odd part first.
__device__ __forceinline__ void inv32_half(const int (&c)[32], int p, const int* __restrict__ tab, int (&lo)[8],
                                           int (&hi)[8]) {
    const int* f = tab + 256 + p * 128;
    int o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {  // n = 8p + i
        int acc = 0;
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
            const int4 t = lds_coef4(f + i * 16 + j);
            acc += t.x * c[2 * j + 1] + t.y * c[2 * j + 3] + t.z * c[2 * j + 5] + t.w * c[2 * j + 7];
        }
        o[i] = acc;
    }
    int ce[16], ee[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ce[i] = c[2 * i];
    inv1d<16>(ce, ee);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int en = p ? ee[8 + i] : ee[i];
        lo[i] = en + o[i];
        hi[7 - i] = en - o[i];
    }
}

__device__ __forceinline__ int clip16(int v) { return v < -32768 ? -32768 : (v > 32767 ? 32767 : v); }
__device__ __forceinline__ int clip_pix(int v) { return v < 0 ? 0 : (v > kPixMax ? kPixMax : v); }

// ---------------------------------------------------------------- quantiser
__device__ __forceinline__ int quant_scale(int r) {
    return r == 0 ? 26214 : r == 1 ? 23302 : r == 2 ? 20560 : r == 3 ? 18396 : r == 4 ? 16384 : 14564;
}
__device__ __forceinline__ int level_scale(int r) {
    return r == 0 ? 40 : r == 1 ? 45 : r == 2 ? 51 : r == 3 ? 57 : r == 4 ? 64 : 72;
}

struct QuantParams {
    int qbits;        // 14 + qP/6 + 15 - B - log2N
    int64_t offset;   // 85 << (qbits - 9)
    int64_t qscale;   // forward scale for qP % 6
    int64_t dqscale;  // 16 * levelScale[qP % 6] << (qP / 6)
    int bd;           // B + log2N - 5
    int lmax32;       // |level| <= lmax32: level * dqscale + 2^(bd-1) fits int32
};

__device__ __forceinline__ QuantParams quant_params(int qp, int log2n) {
    QuantParams q;
    int qP = qp + 6 * (kBitDepth - 8);
    q.qbits = 14 + qP / 6 + 15 - kBitDepth - log2n;
    q.offset = (int64_t)85 << (q.qbits - 9);
    q.qscale = quant_scale(qP % 6);
    q.dqscale = ((int64_t)16 * level_scale(qP % 6)) << (qP / 6);
    q.bd = kBitDepth + log2n - 5;
    q.lmax32 = (int)((((int64_t)1 << 31) - 1 - ((int64_t)1 << (q.bd - 1))) / q.dqscale);
    return q;
}

__device__ __forceinline__ int quantize(int c, const QuantParams& q) {
    const unsigned a = c < 0 ? 0u - (unsigned)c : (unsigned)c;
    int64_t m;
    if (a < 65536u) {
        // |c| < 2^16, scale < 2^15, offset < 2^26: the sum fits 32 bits
        m = (int64_t)((a * (unsigned)q.qscale + (unsigned)q.offset) >> q.qbits);
    } else {
        m = ((int64_t)a * q.qscale + q.offset) >> q.qbits;
    }
    if (m > 32767) m = c < 0 ? 32768 : 32767;  // int16 clip of +/- magnitude
    return c < 0 ? -(int)m : (int)m;
}

__device__ __forceinline__ int dequantize(int level, const QuantParams& q) {
    if (level == 0) return 0;  // (0 + 2^(bd-1)) >> bd
    if ((unsigned)(level + q.lmax32) <= 2u * (unsigned)q.lmax32) {
        // the product and the rounding offset fit 32 bits: the same floor
        const int v = (level * (int)q.dqscale + (1 << (q.bd - 1))) >> q.bd;
        return v < -32768 ? -32768 : (v > 32767 ? 32767 : v);
    }
    int64_t v = ((int64_t)level * q.dqscale + ((int64_t)1 << (q.bd - 1))) >> q.bd;
    return v < -32768 ? -32768 : (v > 32767 ? 32767 : (int)v);
}

// ------------------------------------------------------------------ rate
// Length of the Exp-Golomb code of the signed value v (se(v) -> ue(k)).
__device__ __forceinline__ int se_len(int v) {
    unsigned k = v > 0 ? 2u * (unsigned)v - 1u : 2u * (unsigned)(-v);
    return 2 * (31 - __clz((int)(k + 1u))) + 1;
}

// The encoder's per-coefficient step: the level of transform coefficient c
// (quantize), its rate added to `bits` (2 log2N + se_len(level) when the
// level is not 0) and its de-quantised value in `deq`.  (A branch-free form
// with the rate as 65 - 2 clz(|level|) measured slower.)
__device__ __forceinline__ int quant_rate_deq(int c, const QuantParams& q, int L, uint32_t& bits, int& deq) {
    const int lv = quantize(c, q);
    if (lv != 0) bits += (uint32_t)(2 * L + se_len(lv));
    deq = dequantize(lv, q);
    return lv;
}
__device__ __forceinline__ uint32_t mv_cost(int mvx, int mvy, int64_t lambda_mv_fp16) {
    return (uint32_t)((lambda_mv_fp16 * (se_len(mvx) + se_len(mvy)) + 32768) >> 16);
}

// ----------------------------------------------------------- interpolation
// HEVC luma filter tap i (0..7, at offset i - 3) for fractional phase f.
__device__ __forceinline__ int luma_tap(int f, int i) {
    // phase 1: -1 4 -10 58 17 -5 1 0; phase 2: -1 4 -11 40 40 -11 4 -1;
    // phase 3 is phase 1 mirrored.
    if (f == 3) { f = 1; i = 7 - i; }
    if (f == 1) {
        return i == 0 ? -1 : i == 1 ? 4 : i == 2 ? -10 : i == 3 ? 58 : i == 4 ? 17 : i == 5 ? -5 : i == 6 ? 1 : 0;
    }
    return (i == 0 || i == 7) ? -1 : (i == 1 || i == 6) ? 4 : (i == 2 || i == 5) ? -11 : 40;
}

// All 8 taps of phase f (1..3) in registers, so the filter loops multiply by
// register values instead of re-deriving each tap.
__device__ __forceinline__ void luma_taps(int f, int (&t)[8]) {
    if (f == 2) {
        t[0] = -1; t[1] = 4; t[2] = -11; t[3] = 40; t[4] = 40; t[5] = -11; t[6] = 4; t[7] = -1;
    } else if (f == 1) {
        t[0] = -1; t[1] = 4; t[2] = -10; t[3] = 58; t[4] = 17; t[5] = -5; t[6] = 1; t[7] = 0;
    } else {
        t[0] = 0; t[1] = 1; t[2] = -5; t[3] = 17; t[4] = 58; t[5] = -10; t[6] = 4; t[7] = -1;
    }
}

// Intermediate shifts for B = 10: shift1 = B - 8, shift2 = 6, full-sample
// scale 2^(14 - B); weighted-prediction rounding back to B bits.
constexpr int kShift1 = kBitDepth - 8;
constexpr int kShift2 = 6;
constexpr int kShift3 = 14 - kBitDepth;
__device__ __forceinline__ int wp_round(int v) {
    return clip_pix((v + (1 << (kShift3 - 1))) >> kShift3);
}

// Loads of the reference frame.  Within one launch of the per-frame kernels
// the reference is read-only (read-only cache path); in the persistent kernel
// other blocks write it during the launch, so it is read through L2 only.
template <bool kCoherent>
__device__ __forceinline__ int ld_ref(const uint16_t* p) {
    if constexpr (kCoherent) return (int)__ldcg(p);
    else return (int)__ldg(p);
}
template <bool kCoherent>
__device__ __forceinline__ uint4 ld_ref16(const uint4* p) {
    if constexpr (kCoherent) return __ldcg(p);
    else return __ldg(p);
}

}  // namespace xvd
