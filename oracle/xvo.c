/*
 * xvo.c -- CPU oracle (test infrastructure only; see xvo.h).
 *
 * Written as the plain definitions, one loop nest per step, in the order the
 * method runs them:
 *   Sec. 2.1 of the paper: bands are packed three to a video, the last group
 *     padded by repeating its last band; the data are converted to an N-bit
 *     integer video (here 10 bit, per-band min-max).
 *   HEVC-style encoder analysis (the paper drives libx265, Sec. 2.1 and
 *     Table A.1; the analysis stages are stated here from the public H.265
 *     definitions): integer full-search motion estimation with SAD, quarter-pel
 *     refinement with the 8-tap luma filters and Hadamard SATD, the integer
 *     core transform, flat-matrix quantisation and its inverse, reconstruction.
 *   Sec. 2.3: bpppb = bits / (pixels x bands); PSNR against the per-channel
 *     maximum of the original sequence.
 * No blocking, fusion or reordering beyond those definitions.  Compile with
 * -ffp-contract=off: every double operation is rounded on its own.
 */
#include "xvo.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BITDEPTH 10
#define PIXMAX 1023

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int64_t clamp64(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }
/* rs(x, s) = (x + 2^(s-1)) >> s, arithmetic shift (C10). */
static int64_t rshift_round(int64_t x, int s) { return (x + ((int64_t)1 << (s - 1))) >> s; }
static int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

int xvo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void xvo_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ======================= C2/C3: grouping and geometry ======================== */

/* Sec. 2.1: bands go three to a video; the remainder is repeated up to three. */
int xvo_group_count(int bands) { return (bands + 2) / 3; }

int xvo_group_band(int bands, int g, int c) {
    int b = 3 * g + c;
    return b < bands ? b : bands - 1;
}

void xvo_plane_geometry(int H, int W, int ctu, int* Hp, int* Wp) {
    *Hp = (H + ctu - 1) / ctu * ctu;
    *Wp = (W + ctu - 1) / ctu * ctu;
}

static double src_value(const void* src, int dtype, int64_t idx) {
    if (dtype == XVO_F32) return (double)((const float*)src)[idx];
    return (double)((const uint16_t*)src)[idx];
}

/* ========================= C1: min-max quantisation ========================== */

/* Per band: min and max over the finite samples of all T*H*W values.  A band
 * with no finite sample gets min = max = 0. */
void xvo_minmax(const void* src, int dtype, int bands, int T, int H, int W, double* mm,
                int64_t* nan_count) {
    int64_t plane = (int64_t)T * H * W;
    for (int b = 0; b < bands; ++b) {
        double lo = INFINITY, hi = -INFINITY;
        int64_t nn = 0;
        for (int64_t i = 0; i < plane; ++i) {
            double v = src_value(src, dtype, (int64_t)b * plane + i);
            if (!isfinite(v)) { ++nn; continue; }
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        if (nn == plane) { lo = 0.0; hi = 0.0; }
        mm[2 * b] = lo;
        mm[2 * b + 1] = hi;
        if (nan_count) nan_count[b] = nn;
    }
}

/* q = clamp(floor((x - min) * s + 0.5), 0, 1023) with s = 1023 / (max - min),
 * each operation rounded separately; s = 0 for a constant band; non-finite
 * samples map to 0. */
static int quantize_one(double x, double lo, double s) {
    if (!isfinite(x)) return 0;
    double d = x - lo;
    double p = d * s;
    double r = p + 0.5;
    double f = floor(r);
    if (f < 0.0) return 0;
    if (f > (double)PIXMAX) return PIXMAX;
    return (int)f;
}

void xvo_quantize_pack(const void* src, int dtype, int bands, int T, int H, int W, int ctu,
                       const double* mm, uint16_t* planes) {
    int G = xvo_group_count(bands), Hp, Wp;
    xvo_plane_geometry(H, W, ctu, &Hp, &Wp);
    for (int g = 0; g < G; ++g)
        for (int c = 0; c < 3; ++c) {
            int b = xvo_group_band(bands, g, c);
            double lo = mm[2 * b], hi = mm[2 * b + 1];
            double s = (hi > lo) ? (double)PIXMAX / (hi - lo) : 0.0;
            for (int t = 0; t < T; ++t)
                for (int y = 0; y < Hp; ++y)
                    for (int x = 0; x < Wp; ++x) {
                        int sy = y < H ? y : H - 1, sx = x < W ? x : W - 1;
                        int64_t si = (((int64_t)b * T + t) * H + sy) * W + sx;
                        int64_t di = ((((int64_t)g * T + t) * 3 + c) * Hp + y) * Wp + x;
                        planes[di] = (uint16_t)quantize_one(src_value(src, dtype, si), lo, s);
                    }
        }
}

/* ============================ C10: core transform ============================ */

/* The HEVC integer DCT matrix: DC row 64, other rows the scaled cosine table
 * indexed by k(2n+1)(32/N) mod 128 with the cosine's symmetry folded in. */
static const int cos_tab[33] = {64, 90, 90, 90, 89, 88, 87, 85, 83, 82, 80, 78, 75, 73, 70, 67, 64,
                                61, 57, 54, 50, 46, 43, 38, 36, 31, 25, 22, 18, 13, 9,  4,  0};

void xvo_transform_matrix(int N, int32_t* Tm) {
    for (int k = 0; k < N; ++k)
        for (int n = 0; n < N; ++n) {
            int v;
            if (k == 0) {
                v = 64;
            } else {
                int m = (k * (2 * n + 1) * (32 / N)) % 128;
                if (m > 64) m = 128 - m;
                v = (m <= 32) ? cos_tab[m] : -cos_tab[64 - m];
            }
            Tm[k * N + n] = v;
        }
}

/* Forward: rows first, Y = rs(X T^T, log2N + B - 9); then columns,
 * C = rs(T Y, log2N + 6). */
void xvo_fwd_transform(int N, const int32_t* X, int32_t* C) {
    int32_t Tm[32 * 32];
    int64_t Y[32 * 32];
    int L = ilog2(N);
    xvo_transform_matrix(N, Tm);
    for (int y = 0; y < N; ++y)
        for (int k = 0; k < N; ++k) {
            int64_t acc = 0;
            for (int x = 0; x < N; ++x) acc += (int64_t)X[y * N + x] * Tm[k * N + x];
            Y[y * N + k] = rshift_round(acc, L + BITDEPTH - 9);
        }
    for (int k = 0; k < N; ++k)
        for (int u = 0; u < N; ++u) {
            int64_t acc = 0;
            for (int y = 0; y < N; ++y) acc += (int64_t)Tm[k * N + y] * Y[y * N + u];
            C[k * N + u] = (int32_t)rshift_round(acc, L + 6);
        }
}

/* Inverse: columns first, E = clip16(rs(T^T C, 7)); then rows,
 * R = rs(E T, 20 - B). */
void xvo_inv_transform(int N, const int32_t* C, int32_t* R) {
    int32_t Tm[32 * 32];
    int64_t E[32 * 32];
    xvo_transform_matrix(N, Tm);
    for (int y = 0; y < N; ++y)
        for (int u = 0; u < N; ++u) {
            int64_t acc = 0;
            for (int v = 0; v < N; ++v) acc += (int64_t)Tm[v * N + y] * C[v * N + u];
            E[y * N + u] = clamp64(rshift_round(acc, 7), -32768, 32767);
        }
    for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
            int64_t acc = 0;
            for (int u = 0; u < N; ++u) acc += E[y * N + u] * Tm[u * N + x];
            R[y * N + x] = (int32_t)rshift_round(acc, 20 - BITDEPTH);
        }
}

/* =============================== C11: quantiser ============================== */

static const int64_t quant_scale[6] = {26214, 23302, 20560, 18396, 16384, 14564};
static const int64_t dequant_scale[6] = {40, 45, 51, 57, 64, 72};

/* qP = QP + 6(B-8); qbits = 14 + qP/6 + 15 - B - log2N; offset 85/512 of the
 * step; level = sign(c) ((|c| Q + f) >> qbits), clipped to int16. */
int32_t xvo_quant(int32_t c, int qp, int log2N) {
    int qP = qp + 6 * (BITDEPTH - 8);
    int qbits = 14 + qP / 6 + 15 - BITDEPTH - log2N;
    int64_t f = (int64_t)85 << (qbits - 9);
    int64_t a = c < 0 ? -(int64_t)c : (int64_t)c;
    int64_t lv = (a * quant_scale[qP % 6] + f) >> qbits;
    if (c < 0) lv = -lv;
    return (int32_t)clamp64(lv, -32768, 32767);
}

/* Flat scaling list m = 16; bd = B + log2N - 5;
 * d = clip16((level 16 IQ 2^(qP/6) + 2^(bd-1)) >> bd). */
int32_t xvo_dequant(int32_t level, int qp, int log2N) {
    int qP = qp + 6 * (BITDEPTH - 8);
    int bd = BITDEPTH + log2N - 5;
    int64_t v = (int64_t)level * 16 * dequant_scale[qP % 6] * ((int64_t)1 << (qP / 6));
    v = (v + ((int64_t)1 << (bd - 1))) >> bd;
    return (int32_t)clamp64(v, -32768, 32767);
}

/* ============================ C7: motion-vector cost ========================= */

void xvo_lambdas(int qp, int64_t* lambda_fp8, int64_t* lambda_mv_fp16) {
    double lambda = 0.57 * pow(2.0, (qp - 12) / 3.0);
    *lambda_fp8 = llround(256.0 * lambda);
    *lambda_mv_fp16 = llround(65536.0 * sqrt(lambda));
}

/* Length of the 0th-order Exp-Golomb code of the signed value v (se -> ue). */
int xvo_ue_len_se(int v) {
    int64_t k = v > 0 ? 2 * (int64_t)v - 1 : -2 * (int64_t)v;
    int l = 0;
    while (((int64_t)1 << (l + 1)) <= k + 1) ++l; /* l = floor(log2(k+1)) */
    return 2 * l + 1;
}

int xvo_mv_bits(int mvx_q, int mvy_q) { return xvo_ue_len_se(mvx_q) + xvo_ue_len_se(mvy_q); }

uint32_t xvo_mv_cost(int mvx_q, int mvy_q, int64_t lambda_mv_fp16) {
    return (uint32_t)((lambda_mv_fp16 * xvo_mv_bits(mvx_q, mvy_q) + 32768) >> 16);
}

/* ====================== C8: quarter-sample interpolation ===================== */

static const int luma_filter[4][8] = {
    {0, 0, 0, 64, 0, 0, 0, 0},
    {-1, 4, -10, 58, 17, -5, 1, 0},
    {-1, 4, -11, 40, 40, -11, 4, -1},
    {0, 1, -5, 17, 58, -10, 4, -1},
};

static int refpx(const uint16_t* ref, int Hp, int Wp, int y, int x) {
    return ref[clampi(y, 0, Hp - 1) * Wp + clampi(x, 0, Wp - 1)];
}

/* The predicted sample at (x0 + x, y0 + y) for a quarter-sample motion vector:
 * shift1 = B - 8, shift2 = 6, full samples scaled by 2^(14-B), then the
 * default weighted-prediction rounding back to B bits. */
static int interp_sample(const uint16_t* ref, int Hp, int Wp, int xs, int ys, int mvx_q, int mvy_q) {
    int xi = xs + (mvx_q >> 2), yi = ys + (mvy_q >> 2);
    int fx = mvx_q & 3, fy = mvy_q & 3;
    int shift1 = BITDEPTH - 8, shift2 = 6, shift3 = 14 - BITDEPTH;
    int v;
    if (fx == 0 && fy == 0) {
        v = refpx(ref, Hp, Wp, yi, xi) << shift3;
    } else if (fy == 0) {
        int acc = 0;
        for (int i = 0; i < 8; ++i) acc += luma_filter[fx][i] * refpx(ref, Hp, Wp, yi, xi + i - 3);
        v = acc >> shift1;
    } else if (fx == 0) {
        int acc = 0;
        for (int j = 0; j < 8; ++j) acc += luma_filter[fy][j] * refpx(ref, Hp, Wp, yi + j - 3, xi);
        v = acc >> shift1;
    } else {
        int tmp[8];
        for (int j = 0; j < 8; ++j) {
            int acc = 0;
            for (int i = 0; i < 8; ++i)
                acc += luma_filter[fx][i] * refpx(ref, Hp, Wp, yi + j - 3, xi + i - 3);
            tmp[j] = acc >> shift1;
        }
        int acc = 0;
        for (int j = 0; j < 8; ++j) acc += luma_filter[fy][j] * tmp[j];
        v = acc >> shift2;
    }
    int shiftw = 14 - BITDEPTH;
    return clampi((v + (1 << (shiftw - 1))) >> shiftw, 0, PIXMAX);
}

void xvo_interp_block(const uint16_t* ref, int Hp, int Wp, int x0, int y0, int w, int h,
                      int mvx_q, int mvy_q, uint16_t* out) {
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            out[y * w + x] = (uint16_t)interp_sample(ref, Hp, Wp, x0 + x, y0 + y, mvx_q, mvy_q);
}

/* ================================ C9: SATD =================================== */

static int hadamard_entry(int i, int j) { return (__builtin_popcount(i & j) & 1) ? -1 : 1; }

void xvo_hadamard8(const int32_t* d, int32_t* out) {
    int32_t tmp[64];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            int32_t acc = 0;
            for (int k = 0; k < 8; ++k) acc += hadamard_entry(i, k) * d[k * 8 + j];
            tmp[i * 8 + j] = acc;
        }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            int32_t acc = 0;
            for (int k = 0; k < 8; ++k) acc += tmp[i * 8 + k] * hadamard_entry(j, k);
            out[i * 8 + j] = acc;
        }
}

static uint32_t satd_sub(const int32_t* d, int stride, int n) {
    int32_t tmp[64];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int32_t acc = 0;
            for (int k = 0; k < n; ++k) acc += hadamard_entry(i, k) * d[k * stride + j];
            tmp[i * n + j] = acc;
        }
    uint32_t s = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int32_t acc = 0;
            for (int k = 0; k < n; ++k) acc += tmp[i * n + k] * hadamard_entry(j, k);
            s += (uint32_t)(acc < 0 ? -acc : acc);
        }
    return n == 8 ? (s + 2) >> 2 : (s + 1) >> 1;
}

/* Sum over 8x8 sub-blocks (4x4 when a side is not a multiple of 8) of the
 * normalised absolute Hadamard coefficients of the difference d. */
uint32_t xvo_satd(const int32_t* d, int w, int h) {
    int n = (w % 8 == 0 && h % 8 == 0) ? 8 : 4;
    uint32_t s = 0;
    for (int by = 0; by < h; by += n)
        for (int bx = 0; bx < w; bx += n) s += satd_sub(d + by * w + bx, w, n);
    return s;
}

/* ======================== C7: integer full search ============================ */

void xvo_me_int(const uint16_t* cur, const uint16_t* ref, int Hp, int Wp, int ctu, int R,
                int64_t lambda_mv_fp16, int16_t* mv_int, uint32_t* cost_int) {
    int nx = Wp / ctu, ny = Hp / ctu;
#pragma omp parallel for schedule(dynamic)
    for (int pu = 0; pu < nx * ny; ++pu) {
        int x0 = (pu % nx) * ctu, y0 = (pu / nx) * ctu;
        uint64_t best = UINT64_MAX;
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                uint32_t sad = 0;
                for (int y = 0; y < ctu; ++y)
                    for (int x = 0; x < ctu; ++x) {
                        int a = cur[(y0 + y) * Wp + x0 + x];
                        int b = refpx(ref, Hp, Wp, y0 + y + dy, x0 + x + dx);
                        sad += (uint32_t)(a > b ? a - b : b - a);
                    }
                uint64_t J = (uint64_t)sad + xvo_mv_cost(4 * dx, 4 * dy, lambda_mv_fp16);
                uint64_t idx = (uint64_t)(dy + R) * (2 * R + 1) + (dx + R);
                uint64_t key = (J << 32) | idx;
                if (key < best) best = key;
            }
        int idx = (int)(best & 0xffffffffu);
        mv_int[2 * pu] = (int16_t)(idx % (2 * R + 1) - R);
        mv_int[2 * pu + 1] = (int16_t)(idx / (2 * R + 1) - R);
        cost_int[pu] = (uint32_t)(best >> 32);
    }
}

/* ======================== C8: quarter-pel refinement ========================= */

static uint32_t satd_cost(const uint16_t* cur, const uint16_t* ref, int Hp, int Wp, int x0, int y0,
                          int n, int mvx_q, int mvy_q, int64_t lambda_mv_fp16) {
    int32_t d[64 * 64];
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            d[y * n + x] = (int32_t)cur[(y0 + y) * Wp + x0 + x] -
                           interp_sample(ref, Hp, Wp, x0 + x, y0 + y, mvx_q, mvy_q);
    return xvo_satd(d, n, n) + xvo_mv_cost(mvx_q, mvy_q, lambda_mv_fp16);
}

static const int ring_x[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int ring_y[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

void xvo_me_qpel(const uint16_t* cur, const uint16_t* ref, int Hp, int Wp, int ctu,
                 int64_t lambda_mv_fp16, const int16_t* mv_int, int16_t* mv, uint32_t* cost) {
    int nx = Wp / ctu, ny = Hp / ctu;
#pragma omp parallel for schedule(dynamic)
    for (int pu = 0; pu < nx * ny; ++pu) {
        int x0 = (pu % nx) * ctu, y0 = (pu / nx) * ctu;
        int bx = 4 * mv_int[2 * pu], by = 4 * mv_int[2 * pu + 1];
        uint32_t bJ = satd_cost(cur, ref, Hp, Wp, x0, y0, ctu, bx, by, lambda_mv_fp16);
        for (int step = 2; step >= 1; step /= 2) {
            int cx = bx, cy = by;
            for (int k = 0; k < 8; ++k) {
                int mx = cx + step * ring_x[k], my = cy + step * ring_y[k];
                uint32_t J = satd_cost(cur, ref, Hp, Wp, x0, y0, ctu, mx, my, lambda_mv_fp16);
                if (J < bJ) { bJ = J; bx = mx; by = my; }
            }
        }
        mv[2 * pu] = (int16_t)bx;
        mv[2 * pu + 1] = (int16_t)by;
        cost[pu] = bJ;
    }
}

/* ============ C4/C11/C12/C13: transform, quantise, reconstruct ============== */

/* One CU at (x0, y0) from its prediction pred [3][ctu][ctu]: for each allowed
 * TU size (ascending) the residual of every TU of every channel is
 * transformed (C10), quantised and dequantised (C11), inverse transformed and
 * added back; the size with the least J (C12) is kept: its reconstruction and
 * levels are written, *bestL_out = its log2 size, and the result is its bits
 * (per TU and channel one coded-block flag plus the levels' bits, C13). */
static uint64_t code_cu(const uint16_t* cur, int64_t plane, int Wp, int x0, int y0, int ctu,
                        const int32_t* pred, unsigned tu_mask, int qp, int64_t lambda_fp8,
                        uint16_t* recon, int16_t* levels, int* bestL_out) {
    int n2 = ctu * ctu;
    int32_t* rec_try = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
    int32_t* lev_try = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
    int32_t* rec_best = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
    int32_t* lev_best = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
    int64_t bestJ = INT64_MAX;
    int bestL = -1;
    uint64_t bestBits = 0;
    for (int L = 2; L <= 5; ++L) {
        int N = 1 << L;
        if (!(tu_mask & (1u << L)) || N > ctu) continue;
        uint64_t sse = 0, bits = 0;
        int32_t X[32 * 32], C[32 * 32], D[32 * 32], Rr[32 * 32];
        for (int c = 0; c < 3; ++c)
            for (int ty = 0; ty < ctu; ty += N)
                for (int tx = 0; tx < ctu; tx += N) {
                    for (int y = 0; y < N; ++y)
                        for (int x = 0; x < N; ++x) {
                            int yy = ty + y, xx = tx + x;
                            X[y * N + x] = (int32_t)cur[c * plane + (y0 + yy) * Wp + x0 + xx] -
                                           pred[c * n2 + yy * ctu + xx];
                        }
                    xvo_fwd_transform(N, X, C);
                    uint64_t tb = 1; /* coded-block flag */
                    for (int i = 0; i < N * N; ++i) {
                        int32_t lv = xvo_quant(C[i], qp, L);
                        lev_try[c * n2 + (ty + i / N) * ctu + tx + i % N] = lv;
                        if (lv != 0) tb += (uint64_t)(2 * L + xvo_ue_len_se(lv));
                        D[i] = xvo_dequant(lv, qp, L);
                    }
                    bits += tb;
                    xvo_inv_transform(N, D, Rr);
                    for (int y = 0; y < N; ++y)
                        for (int x = 0; x < N; ++x) {
                            int yy = ty + y, xx = tx + x;
                            int r = clampi(pred[c * n2 + yy * ctu + xx] + Rr[y * N + x], 0, PIXMAX);
                            rec_try[c * n2 + yy * ctu + xx] = r;
                            int e = (int)cur[c * plane + (y0 + yy) * Wp + x0 + xx] - r;
                            sse += (uint64_t)((int64_t)e * e);
                        }
                }
        /* C12: J = (SSE << 8) + lambda_fp8 * bits; ascending N, ties to the
         * larger N. */
        int64_t J = (int64_t)(sse << 8) + lambda_fp8 * (int64_t)bits;
        if (J <= bestJ) {
            bestJ = J;
            bestL = L;
            bestBits = bits;
            memcpy(rec_best, rec_try, sizeof(int32_t) * 3 * (size_t)n2);
            memcpy(lev_best, lev_try, sizeof(int32_t) * 3 * (size_t)n2);
        }
    }
    for (int c = 0; c < 3; ++c)
        for (int y = 0; y < ctu; ++y)
            for (int x = 0; x < ctu; ++x) {
                int64_t o = c * plane + (int64_t)(y0 + y) * Wp + x0 + x;
                recon[o] = (uint16_t)rec_best[c * n2 + y * ctu + x];
                if (levels) levels[o] = (int16_t)lev_best[c * n2 + y * ctu + x];
            }
    *bestL_out = bestL;
    free(rec_try); free(lev_try); free(rec_best); free(lev_best);
    return bestBits;
}

uint64_t xvo_tqr_frame(const uint16_t* cur, const uint16_t* ref, const int16_t* mv, int Hp, int Wp,
                       int ctu, unsigned tu_mask, int qp, int64_t lambda_fp8, uint16_t* recon,
                       int16_t* levels, uint8_t* tu_log2, uint64_t* cu_bits) {
    int nx = Wp / ctu, ny = Hp / ctu, ncu = nx * ny;
    int64_t plane = (int64_t)Hp * Wp;
    uint64_t* bits_per_cu = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)ncu);
#pragma omp parallel for schedule(dynamic)
    for (int cu = 0; cu < ncu; ++cu) {
        int x0 = (cu % nx) * ctu, y0 = (cu / nx) * ctu;
        int n2 = ctu * ctu;
        int32_t* pred = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
        int mvx = ref ? mv[2 * cu] : 0, mvy = ref ? mv[2 * cu + 1] : 0;
        /* C4: frame 0 is predicted by the flat value 2^(B-1); later frames by
         * motion compensation from the previous reconstruction, all channels
         * sharing channel 0's vector (C5). */
        for (int c = 0; c < 3; ++c)
            for (int y = 0; y < ctu; ++y)
                for (int x = 0; x < ctu; ++x)
                    pred[c * n2 + y * ctu + x] =
                        ref ? interp_sample(ref + c * plane, Hp, Wp, x0 + x, y0 + y, mvx, mvy)
                            : (1 << (BITDEPTH - 1));
        int bestL;
        uint64_t bestBits = code_cu(cur, plane, Wp, x0, y0, ctu, pred, tu_mask, qp, lambda_fp8, recon, levels,
                                    &bestL);
        if (tu_log2) tu_log2[cu] = (uint8_t)bestL;
        /* C13: 2 bits for the TU size, the motion vector (none in frame 0),
         * then the coded TUs. */
        bits_per_cu[cu] = 2 + (ref ? (uint64_t)xvo_mv_bits(mvx, mvy) : 0) + bestBits;
        free(pred);
    }
    uint64_t total = 0;
    for (int cu = 0; cu < ncu; ++cu) {
        total += bits_per_cu[cu];
        if (cu_bits) cu_bits[cu] = bits_per_cu[cu];
    }
    free(bits_per_cu);
    return total;
}

/* ================= Intra prediction of frame 0 (option XVO_INTRA) ================ */

/* The H.265 intra prediction of an N x N block (N = the CU size here, reading
 * R4: one prediction per CU from the CU's neighbours, the TU split applying to
 * the residual only), from its reference samples: left[y] = p[-1][y] and
 * top[x] = p[x][-1] for 0 <= x, y < 2N, tl = p[-1][-1].  Mode 0 planar, 1 DC,
 * 2..34 angular with the standard's angle per mode; no reference smoothing
 * and no boundary filters (reading R4). */
static const int intra_angle[35] = {0,   0,   32,  26,  21,  17,  13,  9,  5,  2,  0,  -2,
                                    -5,  -9,  -13, -17, -21, -26, -32, -26, -21, -17, -13, -9,
                                    -5,  -2,  0,   2,   5,   9,   13,  17,  21,  26,  32};

int xvo_intra_angle(int mode) { return mode >= 2 && mode <= 34 ? intra_angle[mode] : 0; }

/* 256 * 32 / angle rounded to the nearest integer, for the negative angles */
int xvo_intra_inv_angle(int angle) {
    switch (angle) {
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

void xvo_intra_pred(const int32_t* left, const int32_t* top, int32_t tl, int N, int mode, int32_t* out) {
    int L = ilog2(N);
    if (mode == 0) { /* planar */
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x)
                out[y * N + x] = ((N - 1 - x) * left[y] + (x + 1) * top[N] + (N - 1 - y) * top[x] +
                                  (y + 1) * left[N] + N) >> (L + 1);
        return;
    }
    if (mode == 1) { /* DC */
        int sum = N;
        for (int i = 0; i < N; ++i) sum += top[i] + left[i];
        for (int i = 0; i < N * N; ++i) out[i] = sum >> (L + 1);
        return;
    }
    /* angular: a main reference along the prediction direction, ref[k] for
     * -N <= k <= 2N (stored at refbuf[k + N]); vertical modes (>= 18) read
     * the top row, horizontal ones the left column */
    int angle = intra_angle[mode];
    int vertical = mode >= 18;
    const int32_t* main_side = vertical ? top : left;
    const int32_t* other_side = vertical ? left : top;
    int32_t refbuf[3 * 64 + 1];
    int32_t* ref = refbuf + N;
    ref[0] = tl;
    for (int k = 1; k <= N; ++k) ref[k] = main_side[k - 1];
    if (angle < 0) {
        int last = (N * angle) >> 5;
        if (last < -1) {
            int inv = xvo_intra_inv_angle(angle);
            for (int k = last; k <= -1; ++k) ref[k] = other_side[-1 + ((k * inv + 128) >> 8)];
        }
    } else {
        for (int k = N + 1; k <= 2 * N; ++k) ref[k] = main_side[k - 1];
    }
    for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
            int pos = vertical ? y : x, along = vertical ? x : y;
            int idx = ((pos + 1) * angle) >> 5, fact = ((pos + 1) * angle) & 31;
            int v = fact ? ((32 - fact) * ref[along + idx + 1] + fact * ref[along + idx + 2] + 16) >> 5
                         : ref[along + idx + 1];
            out[y * N + x] = v;
        }
}

/* The 4N + 1 reference samples of the CU at (x0, y0) from one reconstructed
 * plane: a sample is available when it lies inside the plane and in a CU
 * coded before this one in raster order (so the left, top-left, top and
 * top-right neighbours can be, the below-left never).  Unavailable samples are
 * substituted as H.265 does: in the scan from p[-1][2N-1] up the left column
 * to p[-1][-1] and along the top row to p[2N-1][-1], a missing first sample
 * takes the first available one, every other missing sample its predecessor;
 * with none available all are 2^(B-1). */
void xvo_intra_refs(const uint16_t* plane, int Hp, int Wp, int ctu, int x0, int y0, int32_t* left, int32_t* top,
                    int32_t* tl) {
    int N = ctu, M = 4 * N + 1;
    int32_t sv[4 * 64 + 1];
    int av[4 * 64 + 1];
    int any = 0;
    for (int i = 0; i < M; ++i) {
        int x, y;
        if (i < 2 * N) { x = x0 - 1; y = y0 + 2 * N - 1 - i; }
        else if (i == 2 * N) { x = x0 - 1; y = y0 - 1; }
        else { x = x0 + (i - 2 * N - 1); y = y0 - 1; }
        int in = x >= 0 && y >= 0 && x < Wp && y < Hp;
        int coded = in && ((y / ctu < y0 / ctu) || (y / ctu == y0 / ctu && x / ctu < x0 / ctu));
        av[i] = coded;
        sv[i] = coded ? plane[(int64_t)y * Wp + x] : 0;
        any |= coded;
    }
    if (!any) {
        for (int i = 0; i < M; ++i) sv[i] = 1 << (BITDEPTH - 1);
    } else {
        if (!av[0]) {
            int k = 1;
            while (!av[k]) ++k;
            sv[0] = sv[k];
        }
        for (int i = 1; i < M; ++i)
            if (!av[i]) sv[i] = sv[i - 1];
    }
    for (int j = 0; j < 2 * N; ++j) left[j] = sv[2 * N - 1 - j];
    *tl = sv[2 * N];
    for (int j = 0; j < 2 * N; ++j) top[j] = sv[2 * N + 1 + j];
}

/* Frame 0 with intra prediction, CUs in raster order: the mode with the least
 * SATD (C9) of channel 0's residual (ties: the lower mode) predicts all three
 * channels; then the CU is coded like an inter CU.  mode_mv[cu] = (mode, 0).
 * Rate proxy per CU: 2 (TU size) + 6 (mode) + the coded TUs. */
uint64_t xvo_intra_frame(const uint16_t* cur, int Hp, int Wp, int ctu, unsigned tu_mask, int qp,
                         int64_t lambda_fp8, uint16_t* recon, int16_t* levels, uint8_t* tu_log2, int16_t* mode_mv,
                         uint64_t* cu_bits) {
    int nx = Wp / ctu, ny = Hp / ctu, N = ctu, n2 = N * N;
    int64_t plane = (int64_t)Hp * Wp;
    int32_t* pred = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
    int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)n2);
    int32_t left[3][128], top[3][128], tl[3];
    uint64_t total = 0;
    for (int cu = 0; cu < nx * ny; ++cu) {
        int x0 = (cu % nx) * N, y0 = (cu / nx) * N;
        for (int c = 0; c < 3; ++c) xvo_intra_refs(recon + c * plane, Hp, Wp, ctu, x0, y0, left[c], top[c], &tl[c]);
        int best = 0;
        uint32_t bestS = 0xffffffffu;
        for (int m = 0; m < 35; ++m) {
            xvo_intra_pred(left[0], top[0], tl[0], N, m, pred);
            for (int y = 0; y < N; ++y)
                for (int x = 0; x < N; ++x) d[y * N + x] = (int32_t)cur[(int64_t)(y0 + y) * Wp + x0 + x] - pred[y * N + x];
            uint32_t sa = xvo_satd(d, N, N);
            if (sa < bestS) { bestS = sa; best = m; }
        }
        for (int c = 0; c < 3; ++c) xvo_intra_pred(left[c], top[c], tl[c], N, best, pred + c * n2);
        int bestL;
        uint64_t b = code_cu(cur, plane, Wp, x0, y0, ctu, pred, tu_mask, qp, lambda_fp8, recon, levels, &bestL);
        if (tu_log2) tu_log2[cu] = (uint8_t)bestL;
        if (mode_mv) { mode_mv[2 * cu] = (int16_t)best; mode_mv[2 * cu + 1] = 0; }
        uint64_t cb = 2 + 6 + b;
        if (cu_bits) cu_bits[cu] = cb;
        total += cb;
    }
    free(pred); free(d);
    return total;
}

/* ==================== In-loop deblocking (option XVO_DEBLOCK) ===================== */

/* The standard's beta' (QP 0..51) and tC' (QP 0..53) tables, for 8-bit
 * samples; scaled by 2^(B-8). */
static const int deblock_beta[52] = {0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  6,  7,
                                     8,  9,  10, 11, 12, 13, 14, 15, 16, 17, 18, 20, 22, 24, 26, 28, 30, 32,
                                     34, 36, 38, 40, 42, 44, 46, 48, 50, 52, 54, 56, 58, 60, 62, 64};
static const int deblock_tc[54] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,  1,  1,  1,  1,  1,  1,  1,  1, 1,
                                   2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 5, 5, 6, 6, 7, 8, 9, 10, 11, 13, 14, 16, 18, 20, 22, 24};

void xvo_deblock_params(int qp, int bs, int* beta, int* tc) {
    *beta = deblock_beta[clampi(qp, 0, 51)] << (BITDEPTH - 8);
    *tc = bs > 0 ? deblock_tc[clampi(qp + 2 * (bs - 1), 0, 53)] << (BITDEPTH - 8) : 0;
}

/* One 4-sample edge segment: s[k][i] is sample i of line k across the edge,
 * i = 0..3 the p side (p3, p2, p1, p0) and 4..7 the q side (q0..q3). */
void xvo_deblock_segment(int32_t s[4][8], int bs, int qp) {
    int beta, tc;
    xvo_deblock_params(qp, bs, &beta, &tc);
#define P(k, i) s[k][3 - (i)]
#define Q(k, i) s[k][4 + (i)]
    int dp0 = abs(P(0, 2) - 2 * P(0, 1) + P(0, 0)), dp3 = abs(P(3, 2) - 2 * P(3, 1) + P(3, 0));
    int dq0 = abs(Q(0, 2) - 2 * Q(0, 1) + Q(0, 0)), dq3 = abs(Q(3, 2) - 2 * Q(3, 1) + Q(3, 0));
    int d = dp0 + dq0 + dp3 + dq3;
    if (bs == 0 || d >= beta) return;
    int strong = 1;
    for (int k = 0; k < 4; k += 3) {
        int dpq = k == 0 ? dp0 + dq0 : dp3 + dq3;
        if (!(2 * dpq < (beta >> 2) && abs(P(k, 3) - P(k, 0)) + abs(Q(k, 0) - Q(k, 3)) < (beta >> 3) &&
              abs(P(k, 0) - Q(k, 0)) < ((5 * tc + 1) >> 1)))
            strong = 0;
    }
    int dEp = (dp0 + dp3) < ((beta + (beta >> 1)) >> 3), dEq = (dq0 + dq3) < ((beta + (beta >> 1)) >> 3);
    for (int k = 0; k < 4; ++k) {
        int p0 = P(k, 0), p1 = P(k, 1), p2 = P(k, 2), p3 = P(k, 3);
        int q0 = Q(k, 0), q1 = Q(k, 1), q2 = Q(k, 2), q3 = Q(k, 3);
        if (strong) {
            P(k, 0) = clampi((p2 + 2 * p1 + 2 * p0 + 2 * q0 + q1 + 4) >> 3, p0 - 2 * tc, p0 + 2 * tc);
            P(k, 1) = clampi((p2 + p1 + p0 + q0 + 2) >> 2, p1 - 2 * tc, p1 + 2 * tc);
            P(k, 2) = clampi((2 * p3 + 3 * p2 + p1 + p0 + q0 + 4) >> 3, p2 - 2 * tc, p2 + 2 * tc);
            Q(k, 0) = clampi((p1 + 2 * p0 + 2 * q0 + 2 * q1 + q2 + 4) >> 3, q0 - 2 * tc, q0 + 2 * tc);
            Q(k, 1) = clampi((p0 + q0 + q1 + q2 + 2) >> 2, q1 - 2 * tc, q1 + 2 * tc);
            Q(k, 2) = clampi((p0 + q0 + q1 + 3 * q2 + 2 * q3 + 4) >> 3, q2 - 2 * tc, q2 + 2 * tc);
        } else {
            int delta = (9 * (q0 - p0) - 3 * (q1 - p1) + 8) >> 4;
            if (abs(delta) >= tc * 10) continue;
            delta = clampi(delta, -tc, tc);
            P(k, 0) = clampi(p0 + delta, 0, PIXMAX);
            Q(k, 0) = clampi(q0 - delta, 0, PIXMAX);
            if (dEp) P(k, 1) = clampi(p1 + clampi((((p2 + p0 + 1) >> 1) - p1 + delta) >> 1, -(tc >> 1), tc >> 1), 0, PIXMAX);
            if (dEq) Q(k, 1) = clampi(q1 + clampi((((q2 + q0 + 1) >> 1) - q1 - delta) >> 1, -(tc >> 1), tc >> 1), 0, PIXMAX);
        }
    }
#undef P
#undef Q
}

/* Boundary strength of the edge between the samples (xp, yp) and (xq, yq) of
 * neighbouring CUs or TUs (reading R5): 2 when intra; 1 when either TU has a
 * non-zero level in any channel, or the two CUs' vectors differ by 4 quarter
 * samples or more in x or y; else 0. */
static int deblock_bs(int xp, int yp, int xq, int yq, int Hp, int Wp, int ctu, const uint8_t* tu_log2,
                      const int16_t* levels, const int16_t* mv, int intra) {
    if (intra) return 2;
    int nx = Wp / ctu;
    int64_t plane = (int64_t)Hp * Wp;
    int cuP = (yp / ctu) * nx + xp / ctu, cuQ = (yq / ctu) * nx + xq / ctu;
    int pts[2][2] = {{xp, yp}, {xq, yq}};
    int cus[2] = {cuP, cuQ};
    for (int s2 = 0; s2 < 2; ++s2) {
        int TS = 1 << tu_log2[cus[s2]];
        int tx = pts[s2][0] / TS * TS, ty = pts[s2][1] / TS * TS;
        for (int c = 0; c < 3; ++c)
            for (int y = 0; y < TS; ++y)
                for (int x = 0; x < TS; ++x)
                    if (levels[c * plane + (int64_t)(ty + y) * Wp + tx + x] != 0) return 1;
    }
    if (cuP != cuQ && (abs(mv[2 * cuP] - mv[2 * cuQ]) >= 4 || abs(mv[2 * cuP + 1] - mv[2 * cuQ + 1]) >= 4))
        return 1;
    return 0;
}

/* An edge at sample position e (x for vertical edges, y for horizontal ones)
 * is filtered when it lies on the 8 x 8 grid inside the plane and is a CU
 * boundary or a boundary of the TUs of the CU that contains sample e. */
static int deblock_is_edge(int e, int other, int vertical, int Wp, int ctu, const uint8_t* tu_log2) {
    if (e % 8 != 0 || e == 0) return 0;
    if (e % ctu == 0) return 1;
    int nx = Wp / ctu;
    int x = vertical ? e : other, y = vertical ? other : e;
    int TS = 1 << tu_log2[(y / ctu) * nx + x / ctu];
    return e % TS == 0;
}

/* Deblocks one reconstructed frame [3][Hp][Wp] in place (reading R5): the
 * standard's luma filter on all three channels, every vertical edge of the
 * plane first, then every horizontal edge on the result; 4-sample segments;
 * the boundary strength decided once per segment for the three channels. */
void xvo_deblock_frame(uint16_t* rec, int Hp, int Wp, int ctu, int qp, const uint8_t* tu_log2,
                       const int16_t* levels, const int16_t* mv, int intra) {
    int64_t plane = (int64_t)Hp * Wp;
    for (int pass = 0; pass < 2; ++pass) {
        int vertical = pass == 0;
        int E = vertical ? Wp : Hp, O = vertical ? Hp : Wp;
        for (int e = 8; e < E; e += 8)
            for (int o = 0; o < O; o += 4) {
                if (!deblock_is_edge(e, o, vertical, Wp, ctu, tu_log2)) continue;
                int bs = vertical ? deblock_bs(e - 1, o, e, o, Hp, Wp, ctu, tu_log2, levels, mv, intra)
                                  : deblock_bs(o, e - 1, o, e, Hp, Wp, ctu, tu_log2, levels, mv, intra);
                if (bs == 0) continue;
                for (int c = 0; c < 3; ++c) {
                    int32_t s[4][8];
                    for (int k = 0; k < 4; ++k)
                        for (int i = 0; i < 8; ++i) {
                            int64_t at = vertical ? (int64_t)(o + k) * Wp + (e - 4 + i) : (int64_t)(e - 4 + i) * Wp + (o + k);
                            s[k][i] = rec[c * plane + at];
                        }
                    xvo_deblock_segment(s, bs, qp);
                    for (int k = 0; k < 4; ++k)
                        for (int i = 0; i < 8; ++i) {
                            int64_t at = vertical ? (int64_t)(o + k) * Wp + (e - 4 + i) : (int64_t)(e - 4 + i) * Wp + (o + k);
                            rec[c * plane + at] = (uint16_t)s[k][i];
                        }
                }
            }
    }
}

/* ===================== C4: the closed-loop chain per group ==================== */

int xvo_encode_planes_ex(const uint16_t* planes, int G, int T, int Hp, int Wp, int ctu, int R,
                         unsigned tu_mask, int qp, unsigned flags, uint16_t* recon, int16_t* mv, uint32_t* cost,
                         int16_t* mv_int, uint32_t* cost_int, int16_t* levels, uint8_t* tu_log2,
                         uint64_t* bits) {
    int64_t lf8, lmv;
    xvo_lambdas(qp, &lf8, &lmv);
    int npu = (Hp / ctu) * (Wp / ctu);
    int64_t fsz = 3 * (int64_t)Hp * Wp;
    int16_t* mvi = (int16_t*)malloc(sizeof(int16_t) * 2 * (size_t)npu);
    uint32_t* ci = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)npu);
    int16_t* mvq = (int16_t*)malloc(sizeof(int16_t) * 2 * (size_t)npu);
    uint32_t* cq = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)npu);
    /* levels and TU sizes are needed by the deblocking filter even when the
     * caller does not ask for them */
    int16_t* lev_f = levels ? levels : (int16_t*)malloc(sizeof(int16_t) * (size_t)(G * T) * (size_t)fsz);
    uint8_t* tu_f = tu_log2 ? tu_log2 : (uint8_t*)malloc((size_t)G * T * (size_t)npu);
    for (int g = 0; g < G; ++g)
        for (int t = 0; t < T; ++t) {
            int64_t f = (int64_t)g * T + t;
            const uint16_t* cur = planes + f * fsz;
            const uint16_t* ref = t > 0 ? recon + (f - 1) * fsz : NULL;
            if (ref) {
                xvo_me_int(cur, ref, Hp, Wp, ctu, R, lmv, mvi, ci);
                xvo_me_qpel(cur, ref, Hp, Wp, ctu, lmv, mvi, mvq, cq);
            } else {
                memset(mvi, 0, sizeof(int16_t) * 2 * (size_t)npu);
                memset(ci, 0, sizeof(uint32_t) * (size_t)npu);
                memset(mvq, 0, sizeof(int16_t) * 2 * (size_t)npu);
                memset(cq, 0, sizeof(uint32_t) * (size_t)npu);
            }
            if (!ref && (flags & XVO_INTRA)) /* frame 0 intra: its modes take the vectors' place */
                bits[f] = xvo_intra_frame(cur, Hp, Wp, ctu, tu_mask, qp, lf8, recon + f * fsz, lev_f + f * fsz,
                                          tu_f + f * npu, mvq, NULL);
            else
                bits[f] = xvo_tqr_frame(cur, ref, mvq, Hp, Wp, ctu, tu_mask, qp, lf8, recon + f * fsz,
                                        lev_f + f * fsz, tu_f + f * npu, NULL);
            if (mv) memcpy(mv + f * 2 * npu, mvq, sizeof(int16_t) * 2 * (size_t)npu);
            if (cost) memcpy(cost + f * npu, cq, sizeof(uint32_t) * (size_t)npu);
            if (mv_int) memcpy(mv_int + f * 2 * npu, mvi, sizeof(int16_t) * 2 * (size_t)npu);
            if (cost_int) memcpy(cost_int + f * npu, ci, sizeof(uint32_t) * (size_t)npu);
            /* in-loop deblocking: the deblocked frame is the next frame's
             * reference and the output */
            if (flags & XVO_DEBLOCK)
                xvo_deblock_frame(recon + f * fsz, Hp, Wp, ctu, qp, tu_f + f * npu, lev_f + f * fsz, mvq,
                                  !ref && (flags & XVO_INTRA));
        }
    free(mvi); free(ci); free(mvq); free(cq);
    if (!levels) free(lev_f);
    if (!tu_log2) free(tu_f);
    return 0;
}

int xvo_encode_planes(const uint16_t* planes, int G, int T, int Hp, int Wp, int ctu, int R, unsigned tu_mask,
                      int qp, uint16_t* recon, int16_t* mv, uint32_t* cost, int16_t* mv_int, uint32_t* cost_int,
                      int16_t* levels, uint8_t* tu_log2, uint64_t* bits) {
    return xvo_encode_planes_ex(planes, G, T, Hp, Wp, ctu, R, tu_mask, qp, 0u, recon, mv, cost, mv_int, cost_int,
                                levels, tu_log2, bits);
}

/* ======================= Decoder (the inverse of C4..C13) ===================== */

/* One frame of one group from its coded data: per CU the same prediction as
 * the encoder (C4: flat 2^(B-1) in frame 0, else channel 0's vector applied
 * to all three channels of the previous reconstruction, C5/C6), then per TU
 * of the CU's chosen size the dequantised levels (C11), the inverse
 * transform (C10) and recon = clip(pred + r, 0, 1023).  Returns the frame's
 * rate proxy recomputed from the levels (C13), which must equal the
 * encoder's. */
uint64_t xvo_decode_frame(const int16_t* levels, const uint16_t* ref, const int16_t* mv,
                          const uint8_t* tu_log2, int Hp, int Wp, int ctu, int qp, uint16_t* recon) {
    int nx = Wp / ctu, ny = Hp / ctu, ncu = nx * ny;
    int64_t plane = (int64_t)Hp * Wp;
    uint64_t* bits_per_cu = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)ncu);
#pragma omp parallel for schedule(dynamic)
    for (int cu = 0; cu < ncu; ++cu) {
        int x0 = (cu % nx) * ctu, y0 = (cu / nx) * ctu;
        int mvx = ref ? mv[2 * cu] : 0, mvy = ref ? mv[2 * cu + 1] : 0;
        int L = tu_log2[cu], N = 1 << L;
        uint64_t bits = 2 + (ref ? (uint64_t)xvo_mv_bits(mvx, mvy) : 0);
        int32_t D[32 * 32], Rr[32 * 32];
        for (int c = 0; c < 3; ++c)
            for (int ty = 0; ty < ctu; ty += N)
                for (int tx = 0; tx < ctu; tx += N) {
                    uint64_t tb = 1; /* coded-block flag */
                    for (int y = 0; y < N; ++y)
                        for (int x = 0; x < N; ++x) {
                            int lv = levels[c * plane + (int64_t)(y0 + ty + y) * Wp + x0 + tx + x];
                            if (lv != 0) tb += (uint64_t)(2 * L + xvo_ue_len_se(lv));
                            D[y * N + x] = xvo_dequant(lv, qp, L);
                        }
                    bits += tb;
                    xvo_inv_transform(N, D, Rr);
                    for (int y = 0; y < N; ++y)
                        for (int x = 0; x < N; ++x) {
                            int xs = x0 + tx + x, ys = y0 + ty + y;
                            int pred = ref ? interp_sample(ref + c * plane, Hp, Wp, xs, ys, mvx, mvy)
                                           : (1 << (BITDEPTH - 1));
                            recon[c * plane + (int64_t)ys * Wp + xs] =
                                (uint16_t)clampi(pred + Rr[y * N + x], 0, PIXMAX);
                        }
                }
        bits_per_cu[cu] = bits;
    }
    uint64_t total = 0;
    for (int cu = 0; cu < ncu; ++cu) total += bits_per_cu[cu];
    free(bits_per_cu);
    return total;
}

/* Frame 0 decoded with intra prediction (the inverse of xvo_intra_frame):
 * CUs in raster order, each predicted from its decoded neighbours with the
 * mode mode_mv[cu][0] (clamped to 0..34), then its TUs as in
 * xvo_decode_frame.  Returns the rate proxy, 2 + 6 + the coded TUs per CU. */
uint64_t xvo_decode_intra_frame(const int16_t* levels, const int16_t* mode_mv, const uint8_t* tu_log2, int Hp,
                                int Wp, int ctu, int qp, uint16_t* recon) {
    int nx = Wp / ctu, ny = Hp / ctu, n2 = ctu * ctu;
    int64_t plane = (int64_t)Hp * Wp;
    int32_t* pred = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n2);
    int32_t left[128], top[128], tl;
    uint64_t total = 0;
    for (int cu = 0; cu < nx * ny; ++cu) {
        int x0 = (cu % nx) * ctu, y0 = (cu / nx) * ctu;
        int mode = clampi(mode_mv[2 * cu], 0, 34);
        for (int c = 0; c < 3; ++c) {
            xvo_intra_refs(recon + c * plane, Hp, Wp, ctu, x0, y0, left, top, &tl);
            xvo_intra_pred(left, top, tl, ctu, mode, pred + c * n2);
        }
        int L = tu_log2[cu], N = 1 << L;
        uint64_t bits = 2 + 6;
        int32_t D[32 * 32], Rr[32 * 32];
        for (int c = 0; c < 3; ++c)
            for (int ty = 0; ty < ctu; ty += N)
                for (int tx = 0; tx < ctu; tx += N) {
                    uint64_t tb = 1; /* coded-block flag */
                    for (int y = 0; y < N; ++y)
                        for (int x = 0; x < N; ++x) {
                            int lv = levels[c * plane + (int64_t)(y0 + ty + y) * Wp + x0 + tx + x];
                            if (lv != 0) tb += (uint64_t)(2 * L + xvo_ue_len_se(lv));
                            D[y * N + x] = xvo_dequant(lv, qp, L);
                        }
                    bits += tb;
                    xvo_inv_transform(N, D, Rr);
                    for (int y = 0; y < N; ++y)
                        for (int x = 0; x < N; ++x)
                            recon[c * plane + (int64_t)(y0 + ty + y) * Wp + x0 + tx + x] = (uint16_t)clampi(
                                pred[c * n2 + (ty + y) * ctu + tx + x] + Rr[y * N + x], 0, PIXMAX);
                }
        total += bits;
    }
    free(pred);
    return total;
}

/* The whole chain per group, frames in order; with XVO_INTRA frame 0 is
 * decoded with intra prediction, with XVO_DEBLOCK every decoded frame is
 * deblocked before it is the next frame's reference (as the encoder does). */
int xvo_decode_planes_ex(const int16_t* levels, const int16_t* mv, const uint8_t* tu_log2, int G, int T, int Hp,
                         int Wp, int ctu, int qp, unsigned flags, uint16_t* recon, uint64_t* bits) {
    int npu = (Hp / ctu) * (Wp / ctu);
    int64_t fsz = 3 * (int64_t)Hp * Wp;
    for (int g = 0; g < G; ++g)
        for (int t = 0; t < T; ++t) {
            int64_t f = (int64_t)g * T + t;
            int intra = t == 0 && (flags & XVO_INTRA);
            if (intra)
                bits[f] = xvo_decode_intra_frame(levels + f * fsz, mv + f * 2 * npu, tu_log2 + f * npu, Hp, Wp, ctu,
                                                 qp, recon + f * fsz);
            else
                bits[f] = xvo_decode_frame(levels + f * fsz, t > 0 ? recon + (f - 1) * fsz : NULL,
                                           mv + f * 2 * npu, tu_log2 + f * npu, Hp, Wp, ctu, qp,
                                           recon + f * fsz);
            if (flags & XVO_DEBLOCK)
                xvo_deblock_frame(recon + f * fsz, Hp, Wp, ctu, qp, tu_log2 + f * npu, levels + f * fsz,
                                  mv + f * 2 * npu, intra);
        }
    return 0;
}

int xvo_decode_planes(const int16_t* levels, const int16_t* mv, const uint8_t* tu_log2, int G, int T,
                      int Hp, int Wp, int ctu, int qp, uint16_t* recon, uint64_t* bits) {
    return xvo_decode_planes_ex(levels, mv, tu_log2, G, T, Hp, Wp, ctu, qp, 0u, recon, bits);
}

/* The reconstruction back in the cube's units (the inverse of C1/C2): band b
 * (group b/3, channel b%3) over the valid H x W region, x^ = min + q
 * (max - min)/1023 in double (multiply, then add), rounded to float32. */
void xvo_unpack(const uint16_t* recon, int bands, int T, int H, int W, int Hp, int Wp, const double* mm,
                float* dst) {
    for (int b = 0; b < bands; ++b) {
        int g = b / 3, c = b % 3;
        double lo = mm[2 * b], hi = mm[2 * b + 1];
        double delta = (hi - lo) / (double)PIXMAX;
        for (int t = 0; t < T; ++t)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    int q = recon[((((int64_t)g * T + t) * 3 + c) * Hp + y) * Wp + x];
                    double xh = lo + (double)q * delta;
                    dst[(((int64_t)b * T + t) * H + y) * W + x] = (float)xh;
                }
    }
}

/* ============================ SSIM and spectral angle ========================== */

/* The 11-tap Gaussian window of SSIM (sigma 1.5), normalised to sum 1; the 2-D
 * window is the outer product. */
void xvo_ssim_window(double* w) {
    double s = 0.0;
    for (int k = 0; k < 11; ++k) {
        w[k] = exp(-(double)((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5));
        s += w[k];
    }
    for (int k = 0; k < 11; ++k) w[k] /= s;
}

/* Sum of the SSIM map of one image pair over its valid window positions
 * (every 11 x 11 window inside the H x W image), skipping windows with a
 * non-finite sample of X; *nwin += the windows counted.  Local statistics
 * are Gaussian-weighted: mu = sum w x, sigma_x^2 = sum w (x - mu_x)^2,
 * sigma_xy = sum w (x - mu_x)(y - mu_y); C1 = (0.01 L)^2, C2 = (0.03 L)^2. */
double xvo_ssim_image(const double* X, const double* Y, int H, int W, double L, int64_t* nwin) {
    double w[11];
    xvo_ssim_window(w);
    const double C1 = (0.01 * L) * (0.01 * L), C2 = (0.03 * L) * (0.03 * L);
    double sum = 0.0, comp = 0.0;
    for (int i = 0; i + 11 <= H; ++i)
        for (int j = 0; j + 11 <= W; ++j) {
            double mx = 0.0, my = 0.0;
            int finite = 1;
            for (int u = 0; u < 11; ++u)
                for (int v = 0; v < 11; ++v) {
                    double x = X[(int64_t)(i + u) * W + j + v];
                    if (!isfinite(x)) finite = 0;
                    mx += w[u] * w[v] * x;
                    my += w[u] * w[v] * Y[(int64_t)(i + u) * W + j + v];
                }
            if (!finite) continue;
            double sxx = 0.0, syy = 0.0, sxy = 0.0;
            for (int u = 0; u < 11; ++u)
                for (int v = 0; v < 11; ++v) {
                    double dx = X[(int64_t)(i + u) * W + j + v] - mx;
                    double dy = Y[(int64_t)(i + u) * W + j + v] - my;
                    sxx += w[u] * w[v] * dx * dx;
                    syy += w[u] * w[v] * dy * dy;
                    sxy += w[u] * w[v] * dx * dy;
                }
            double v = ((2.0 * mx * my + C1) * (2.0 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2));
            double yk = v - comp, t = sum + yk; /* Kahan */
            comp = (t - sum) - yk;
            sum = t;
            ++*nwin;
        }
    return sum;
}

/* Mean SSIM per real band between the cube and its reconstruction
 * x^ = min + q (max - min)/1023, over every frame; L = max - min of the band
 * (a constant band, L = 0, counts as 1).  NaN when no window fits. */
void xvo_ssim(const void* src, int dtype, int bands, int T, int H, int W, const uint16_t* recon, int Hp, int Wp,
              const double* mm, double* ssim_band) {
    double* X = (double*)malloc(sizeof(double) * (size_t)H * W);
    double* Y = (double*)malloc(sizeof(double) * (size_t)H * W);
    for (int b = 0; b < bands; ++b) {
        int g = b / 3, c = b % 3;
        double lo = mm[2 * b], hi = mm[2 * b + 1], L = hi - lo;
        double delta = L / (double)PIXMAX;
        double sum = 0.0;
        int64_t n = 0;
        for (int t = 0; t < T; ++t) {
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    X[(int64_t)y * W + x] = src_value(src, dtype, (((int64_t)b * T + t) * H + y) * W + x);
                    int q = recon[((((int64_t)g * T + t) * 3 + c) * Hp + y) * Wp + x];
                    Y[(int64_t)y * W + x] = lo + (double)q * delta;
                }
            if (L > 0.0) sum += xvo_ssim_image(X, Y, H, W, L, &n);
        }
        if (L <= 0.0) ssim_band[b] = (H >= 11 && W >= 11) ? 1.0 : NAN;
        else ssim_band[b] = n > 0 ? sum / (double)n : NAN;
    }
    free(X); free(Y);
}

/* Mean spectral angle (radians) over the pixels (t, y, x) of the valid
 * region: the angle between s = (x_b) and s^ = (x^_b) over all bands.  It is
 * evaluated as atan2(|s ^ s^|, <s, s^>) with |s ^ s^|^2 = sum over band pairs
 * i < j of (s_i s^_j - s_j s^_i)^2 (Lagrange's identity), which equals
 * acos(<s, s^> / (|s| |s^|)) and stays accurate for small angles.  Pixels
 * with a non-finite sample or a zero spectrum are skipped; *npix = the pixels
 * counted. */
double xvo_sa(const void* src, int dtype, int bands, int T, int H, int W, const uint16_t* recon, int Hp, int Wp,
              const double* mm, int64_t* npix) {
    double sum = 0.0, comp = 0.0;
    int64_t n = 0;
    double s[64], sh[64];
    if (bands > 64) { if (npix) *npix = 0; return NAN; }
    for (int t = 0; t < T; ++t)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double dot = 0.0, n1 = 0.0, n2 = 0.0;
                int ok = 1;
                for (int b = 0; b < bands; ++b) {
                    int g = b / 3, c = b % 3;
                    double lo = mm[2 * b], hi = mm[2 * b + 1];
                    s[b] = src_value(src, dtype, (((int64_t)b * T + t) * H + y) * W + x);
                    int q = recon[((((int64_t)g * T + t) * 3 + c) * Hp + y) * Wp + x];
                    sh[b] = lo + (double)q * ((hi - lo) / (double)PIXMAX);
                    if (!isfinite(s[b])) ok = 0;
                    dot += s[b] * sh[b];
                    n1 += s[b] * s[b];
                    n2 += sh[b] * sh[b];
                }
                if (!ok || n1 <= 0.0 || n2 <= 0.0) continue;
                double cr = 0.0;
                for (int i = 0; i < bands; ++i)
                    for (int j = i + 1; j < bands; ++j) {
                        double m = s[i] * sh[j] - s[j] * sh[i];
                        cr += m * m;
                    }
                double a = atan2(sqrt(cr), dot);
                double yk = a - comp, tt = sum + yk; /* Kahan */
                comp = (tt - sum) - yk;
                sum = tt;
                ++n;
            }
    if (npix) *npix = n;
    return n > 0 ? sum / (double)n : NAN;
}

/* ============================== C14: PSNR ==================================== */

/* Per real band b (slot: group b/3, channel b%3): x^ = min + q^ (max-min)/1023,
 * MSE over the valid finite samples (Kahan-summed), PSNR = 10 log10(peak^2 /
 * MSE) with peak = max (max - min when max <= 0), +inf when MSE = 0.  Also the
 * exact 10-bit SSE against the quantised original and its PSNR at peak 1023. */
void xvo_psnr(const void* src, int dtype, int bands, int T, int H, int W, const uint16_t* planes,
              const uint16_t* recon, int Hp, int Wp, const double* mm, double* psnr_band,
              double* mse_band, uint64_t* sse10_band, double* psnr10_band) {
    for (int b = 0; b < bands; ++b) {
        int g = b / 3, c = b % 3;
        double lo = mm[2 * b], hi = mm[2 * b + 1];
        double delta = (hi - lo) / (double)PIXMAX;
        double sum = 0.0, comp = 0.0;
        int64_t count = 0;
        uint64_t sse10 = 0;
        for (int t = 0; t < T; ++t)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    int64_t pi = ((((int64_t)g * T + t) * 3 + c) * Hp + y) * Wp + x;
                    int rq = recon[pi];
                    int e10 = (int)planes[pi] - rq;
                    sse10 += (uint64_t)((int64_t)e10 * e10);
                    double xv = src_value(src, dtype, (((int64_t)b * T + t) * H + y) * W + x);
                    if (!isfinite(xv)) continue;
                    double xh = lo + (double)rq * delta;
                    double e = xv - xh;
                    double term = e * e;
                    double yk = term - comp; /* Kahan summation */
                    double tk = sum + yk;
                    comp = (tk - sum) - yk;
                    sum = tk;
                    ++count;
                }
        double mse = count > 0 ? sum / (double)count : 0.0;
        double peak = hi > 0.0 ? hi : hi - lo;
        mse_band[b] = mse;
        psnr_band[b] = mse > 0.0 ? 10.0 * log10(peak * peak / mse) : INFINITY;
        sse10_band[b] = sse10;
        double n = (double)T * H * W;
        psnr10_band[b] = sse10 > 0 ? 10.0 * log10((double)PIXMAX * PIXMAX * n / (double)sse10) : INFINITY;
    }
}
