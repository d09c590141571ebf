/*
 * xv.h -- C ABI of the GPU encoder-analysis library (libxv.so, sm_103a).
 *
 * The library compresses multichannel spatiotemporal cubes the way the paper
 * "Video Compression for Spatiotemporal Earth System Data" (arXiv 2506.19656)
 * does -- bands packed three to a video and coded as 10-bit video -- but
 * stops at the encoder analysis: it computes, bit-exactly and on the GPU,
 * the quantised planes, motion vectors, transform levels, reconstruction,
 * and the PSNR / bits-per-pixel-per-band reductions.  There is no entropy
 * coder; "bits" is the rate proxy defined at xv_transform_quant_recon.
 *
 * Conventions for every call:
 *  - All data pointers are caller-owned.  Unless stated otherwise they are
 *    DEVICE pointers on the context's device.  The library never frees them.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it unless marked "synchronous".
 *  - Every call returns an xv_status; nothing aborts or traps.  On error the
 *    message is available from xv_last_error() (thread-local).
 *  - Plane layout: uint16 [G][T][3][Hp][Wp] holding 10-bit samples, G =
 *    ceil(bands / 3) groups, Hp/Wp = H/W rounded up to the CTU size.
 *    Plane pointers (planes, recon, levels, cur, ref) must be 16-byte
 *    aligned and group strides multiples of 8 samples (the kernels move
 *    16-byte chunks); otherwise the call returns XV_EINVAL.
 *  - Signed right shifts are arithmetic.  Bit depth B = 10.
 */
#ifndef XV_H
#define XV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XV_OK = 0,
    XV_EINVAL = -1,     /* a shape, pointer or parameter is out of range */
    XV_ENOMEM = -2,     /* a device allocation failed */
    XV_EBUDGET = -3,    /* the request does not fit the context's memory budget */
    XV_ETIMEOUT = -4,   /* a device-side dependency wait ran out of time */
    XV_EBUSY = -5,      /* the serving queue is full */
    XV_ECUDA = -6,      /* a CUDA runtime call or kernel launch failed */
    XV_ECANCELLED = -7, /* the serving request was cancelled */
    XV_ENOTFOUND = -8   /* unknown serving ticket */
} xv_status;

typedef enum { XV_F32 = 0, XV_U16 = 1 } xv_dtype;

#define XV_MAX_BANDS 16

/* Encoder parameters of one cube; restates the paper's per-video mapping
 * rules (Sec. 2.1: codec parameters and output bit depth per video). */
typedef struct {
    int bit_depth;          /* 10 (the only depth in scope) */
    int ctu;                /* PU = CU = CTU size: 8, 16, 32 or 64 */
    int search_range;       /* R: integer search over [-R, R]^2, 1..64 */
    unsigned tu_mask;       /* bit k set: TU size 2^k allowed (k = 2..5); >= 1 size <= ctu */
    int qp;                 /* QP_Y in [-12, 51]; qP = qp + 6 (B - 8) */
    int64_t lambda_fp8;     /* round(256 * lambda), lambda = 0.57 * 2^((qp - 12) / 3) */
    int64_t lambda_mv_fp16; /* round(65536 * sqrt(lambda)) */
    unsigned flags;         /* options, 0 by default: XV_INTRA | XV_DEBLOCK (xv_encode_cube only) */
} xv_params;

/* Options beyond the default conventions (flat frame-0 prediction, no loop
 * filter): XV_INTRA codes frame 0 with intra prediction (xv_intra_frame),
 * XV_DEBLOCK deblocks every reconstructed frame before it becomes the next
 * frame's reference and the output (xv_deblock_frame).  xv_encode_cube and
 * xv_decode_frame run them; the batched path, serving and the batched
 * decoder reject them (XV_EINVAL). */
#define XV_INTRA 1u
#define XV_DEBLOCK 2u

typedef struct xv_ctx xv_ctx;

/* ------------------------------------------------------------------ context */

/* Creates a context on `device`.  `mem_budget_bytes` caps the device memory
 * the context itself allocates (scratch, serving buffers); 0 = no cap.
 * Synchronous. */
xv_status xv_create(xv_ctx** ctx, int device, size_t mem_budget_bytes);
/* Frees everything the context allocated.  Synchronous.  NULL is a no-op. */
void xv_destroy(xv_ctx* ctx);
/* Message of the last failing call on this thread ("" if none). */
const char* xv_last_error(void);
const char* xv_status_string(xv_status s);
/* Device bytes the context currently holds. */
size_t xv_ctx_bytes(const xv_ctx* ctx);

/* Fills `p` for (ctu, R, tu_mask, qp) and derives the fixed-point lambdas on
 * the host (the device only sees integers).  XV_EINVAL when ctu is not 8..64
 * power of two, R is outside 1..64, no TU size <= ctu is allowed, a TU bit
 * outside 2..5 is set, or qp is outside [-12, 51]. */
xv_status xv_params_init(xv_params* p, int ctu, int search_range, unsigned tu_mask, int qp);

/* G = ceil(bands / 3), Hp = ceil(H / ctu) * ctu, Wp likewise.  Host only. */
xv_status xv_plane_geometry(int bands, int H, int W, int ctu, int* G, int* Hp, int* Wp);

/* ------------------------------------------------- A1/A2: quantise and pack */

/* Per-band minimum and maximum over the finite samples of a cube (paper
 * Sec. 2.1 converts every band to an N-bit integer video; the per-band range
 * is the metadata needed to undo it).  src: [bands][T][H][W] float32 or
 * uint16.  minmax: device double [bands][2] (min, max), written.  A band
 * without finite samples gets (0, 0).  Uses context scratch. */
xv_status xv_minmax(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                    double* minmax, void* stream);

/* Min-max quantisation to 10 bit and packing three bands to a group (paper
 * Sec. 2.1: the remaining bands of the last group are repeated, e.g.
 * R,G,B | NIR,NIR,NIR).  q = clamp(floor((x - min) s + 0.5), 0, 1023) with
 * s = 1023 / (max - min) in IEEE double (s = 0 for a constant band), each
 * operation rounded separately; non-finite samples give 0.  Planes are
 * padded to the CTU grid by repeating the last row and column.
 * minmax: device double [bands][2]; computed first (as xv_minmax) unless
 * `minmax_fixed` is non-zero, in which case it is read.  planes: device
 * uint16 [G][T][3][Hp][Wp], written. */
xv_status xv_quantize_pack(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                           int ctu, double* minmax, int minmax_fixed, uint16_t* planes, void* stream);

/* ---------------------------------------------- A3/A4: motion estimation */

/* Block motion estimation of one frame for G groups (the paper codes every
 * group with libx265, Sec. 2.1; this is the HEVC-style analysis it runs).
 * Per CTU-sized PU, on channel 0 of each group:
 *  integer full search over (dx, dy) in [-R, R]^2 against `ref` with the
 *  sample coordinates clamped to the plane, J = SAD + mvcost(4dx, 4dy), the
 *  smallest (J, (dy+R)(2R+1) + dx+R) wins; then quarter-sample refinement:
 *  the 8 half-sample neighbours, then the 8 quarter-sample neighbours of the
 *  best, each J = SATD(8x8 Hadamard) + mvcost, replacing the best only when
 *  strictly lower.  mvcost(mx, my) = (lambda_mv_fp16 (|se(mx)| + |se(my)|)
 *  + 2^15) >> 16 with |se| the signed Exp-Golomb code length.
 *  The kernels skip candidates whose lower bound (sum over sub-blocks of
 *  |sum cur - sum ref|, plus mvcost) exceeds the J of a candidate already
 *  evaluated; such a candidate can neither win nor tie, so the result is
 *  that of the full search.
 * cur/ref: device uint16, group g's frame at cur + g * plane_gstride, layout
 *   [3][Hp][Wp] (only channel 0 is read).
 * mv: int16 [G][nPU][2] quarter-sample (x, y); cost: uint32 [G][nPU] (final
 *   J); mv_int/cost_int: the integer-search result (may be NULL).  Group g's
 *   rows start at g * pu_gstride PUs.  nPU = (Hp/ctu)(Wp/ctu), raster order. */
xv_status xv_motion_search(xv_ctx* ctx, const uint16_t* cur, const uint16_t* ref, int G,
                           int64_t plane_gstride, int Hp, int Wp, const xv_params* p, int16_t* mv,
                           uint32_t* cost, int16_t* mv_int, uint32_t* cost_int, int64_t pu_gstride,
                           void* stream);

/* -------------------------- A5..A9: transform, quantise, reconstruct */

/* Transform, quantisation and reconstruction of one frame for G groups.
 * Prediction: ref == NULL (first frame) predicts every sample by 512; else
 * each CU is motion-compensated from `ref` (all 3 channels, the CU's
 * quarter-sample vector, HEVC 8-tap luma filter, default weighted rounding).
 * For every allowed TU size N <= ctu (ascending), the CU is tiled by N x N
 * TUs, each channel's residual goes through the HEVC integer core transform
 * (rows: shift log2N + 1; columns: shift log2N + 6), the flat quantiser
 * (qbits = 14 + qP/6 + 15 - B - log2N, offset 85 << (qbits - 9)), the
 * dequantiser (m = 16, levelScale), the inverse (columns: shift 7 + int16
 * clip; rows: shift 20 - B) and recon = clip(pred + r, 0, 1023).  The size
 * with the least J = (SSE << 8) + lambda_fp8 * bits wins, ties to the larger.
 * Rate proxy per CU: 2 (TU size) + |se(mvx)| + |se(mvy)| (not in frame 0) +
 * per TU and channel 1 + sum over nonzero levels of (2 log2N + |se(level)|).
 * cur/ref/recon: device uint16, group g at + g * plane_gstride, [3][Hp][Wp].
 * mv: int16 [G][nPU][2] at + g * pu_gstride * 2 (ignored when ref == NULL).
 * recon: written (it is the next frame's reference).  levels: int16 in the
 *   plane layout (may be NULL).  tu_log2: uint8 [G][nCU] at + g * pu_gstride
 *   (may be NULL).  bits: uint64, group g's frame total is ADDED to
 *   bits[g * bits_gstride] (zero it first). */
xv_status xv_transform_quant_recon(xv_ctx* ctx, const uint16_t* cur, const uint16_t* ref,
                                   const int16_t* mv, int G, int64_t plane_gstride, int Hp, int Wp,
                                   const xv_params* p, int64_t pu_gstride, uint16_t* recon,
                                   int16_t* levels, uint8_t* tu_log2, uint64_t* bits,
                                   int64_t bits_gstride, void* stream);

/* ----------------------------------------------- A10/A11: PSNR and rate */

/* PSNR per real band (paper Sec. 2.3: peak = the maximum of the original
 * sequence for that band; max - min when max <= 0).  Band b is read from
 * group b/3, channel b%3 of `recon`, de-quantised as min + q (max-min)/1023
 * (q: the sample's low 10 bits; planes hold 10-bit samples), and compared
 * with the finite samples of `src` over the valid H x W region.
 * Also the exact 10-bit SSE against `planes`.  psnr_band, mse_band,
 * sse10_band: HOST arrays [bands] (any may be NULL); psnr_mean: HOST, the
 * mean of the per-band PSNR (+inf when any band is exact).  Synchronous. */
xv_status xv_psnr(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                  const uint16_t* planes, const uint16_t* recon, int Hp, int Wp, const double* minmax,
                  double* psnr_band, double* mse_band, uint64_t* sse10_band, double* psnr_mean,
                  void* stream);

/* The same PSNR reduction for callers that cannot allocate device memory:
 * for example a process whose device memory belongs to another allocator (a
 * framework's caching pool or a fixed budget that raw cudaMalloc would
 * bypass), or a code path that must not call cudaMalloc/cudaFree because
 * those calls can block on the device or fail part-way through a run.  It
 * takes no context and allocates nothing: its scratch is a fixed device
 * array of about 129 KB inside the library, which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart; this
 * is a deployment variant of xv_psnr with identical results.
 *  - Limits: bands <= XV_MAX_BANDS (16); larger requests return XV_EINVAL.
 *  - The first call on each device (with that device current) looks up the
 *    array's device address with cudaGetSymbolAddress and keeps it; make that
 *    first call before any stream capture.
 *  - All calls share the array.  Each call rewrites everything it reads, so
 *    nothing carries over from an earlier call, but calls that overlap on the
 *    GPU (different streams or threads at the same time) race on it.
 * Arguments and outputs as xv_psnr (host outputs; synchronous). */
xv_status xv_psnr_noalloc(const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                          const uint16_t* planes, const uint16_t* recon, int Hp, int Wp,
                          const double* minmax, double* psnr_band, double* mse_band,
                          uint64_t* sse10_band, double* psnr_mean, void* stream);

/* ------------------------------------------------------ whole cubes */

/* One cube.  Device buffers, caller-owned: */
typedef struct {
    const void* src;     /* [bands][T][H][W] float32 or uint16 */
    xv_dtype dtype;
    int bands, T, H, W;  /* bands <= XV_MAX_BANDS */
    xv_params p;
    double* minmax;      /* [bands][2]; computed unless minmax_fixed */
    int minmax_fixed;
    uint16_t* planes;    /* [G][T][3][Hp][Wp] quantised input (written) */
    uint16_t* recon;     /* [G][T][3][Hp][Wp] reconstruction (written) */
    int16_t* mv;         /* [G][T][nPU][2] final vectors, or NULL */
    uint32_t* cost;      /* [G][T][nPU] final J, or NULL */
    int16_t* levels;     /* plane layout, or NULL */
    uint8_t* tu_log2;    /* [G][T][nCU], or NULL */
    uint64_t* bits;      /* [G][T] per-frame rate proxy, or NULL */
} xv_job;

typedef struct {
    xv_status status;
    int bands;
    double psnr_mean;    /* mean over bands of psnr_band */
    double bpppb;        /* total bits / (H W T bands) -- rate proxy, see above */
    uint64_t total_bits;
    double psnr_band[XV_MAX_BANDS];
    double mse_band[XV_MAX_BANDS];
    uint64_t sse10_band[XV_MAX_BANDS];
    double latency_s;    /* serving: arrival to completion */
    int ctu;             /* the CTU size the cube was encoded with (its job's p.ctu) */
    int block_size;      /* execution mode of its encode: persistent block size, 1 = per-frame launches */
} xv_result;

/* Splits a cube's job into one job per 3-band group, each with its own QP
 * (the paper's "PCA - all bands" test, Sec. 3 and Tab. 5: the principal
 * components are packed three to a video and the less important videos are
 * coded at a lower quality).  Group g of `whole` (bands 3g .. 3g + 2, the
 * last group repeating its last band) becomes out[g]: src, minmax, planes,
 * recon, mv, cost, levels, tu_log2 and bits point at group g's part of the
 * whole job's buffers (which keep the whole cube's layout), bands = the
 * group's real bands, and its parameters are xv_params_init(ctu, R, tu_mask,
 * qp[g]) with whole->p's flags.  Encoding the out[] jobs (xv_encode_batch)
 * gives, for every group, exactly the whole job's outputs at that group's
 * QP: groups are independent chains and a band's min/max is its own.
 * qp: HOST [G], G = ceil(bands / 3); out: HOST [G], *njobs = G.  Host only;
 * XV_EINVAL for a malformed job or a QP outside [-12, 51]. */
xv_status xv_split_groups(const xv_job* whole, const int* qp, xv_job* out, int* njobs);

/* Bytes of device scratch a job needs beyond its own buffers. */
size_t xv_job_scratch_bytes(const xv_job* job);

/* Plain path: quantise/pack, then frame by frame one motion-search and one
 * transform launch for all groups, then PSNR.  `result` is a HOST struct.
 * Synchronous (waits for the PSNR read-back). */
xv_status xv_encode_cube(xv_ctx* ctx, const xv_job* job, xv_result* result, void* stream);

/* Batched path: all jobs' frames run in ONE persistent launch per CTU size,
 * scheduled by data flow over a device ready queue of (job, group, frame, PU)
 * items: an item is queued once the previous frame's reconstruction rows it
 * reads are complete, and blocks take queued items in order.  The autotuner
 * also weighs a second execution mode, the per-frame mode: every job's frames
 * as the per-frame motion-search and transform launches of xv_encode_cube,
 * the jobs on up to 16 concurrent streams forked from and joined back to the
 * batch's stream.  The first batch of a given shape on a context tunes: per
 * CTU class every block size (128, 192, 256, 512) with as many resident
 * blocks per SM as fit and with one fewer, and the per-frame mode for the
 * whole batch, each timed as the CUDA graph it would replay (median of three
 * replays after one warm-up); each class keeps its fastest configuration
 * unless the per-frame mode beats their sum (xv_last_batch_config,
 * xv_last_tune_log).  Output is bit-identical to
 * xv_encode_cube for each job, in every mode.  results: HOST [njobs].  Synchronous.  XV_ETIMEOUT if a
 * bounded device wait ran out of time (results then invalid; the context
 * stays usable). */
xv_status xv_encode_batch(xv_ctx* ctx, const xv_job* jobs, int njobs, xv_result* results, void* stream);

/* xv_encode_batch with the cubes coming from HOST memory: for every job whose
 * host_src[i] is not NULL, that host cube ([bands][T][H][W] of the job's
 * dtype, bands T H W elements) is copied into the job's device buffer
 * jobs[i].src, and the batch computes exactly what xv_encode_batch computes
 * (same output, same host results).  With pinned host cubes, in the
 * per-frame mode the copies run on a stream of their own, smallest cube
 * first, and each job's min/max, quantisation and chain start as soon as the
 * copies into its source buffer (its own, or another job's into the same
 * memory) have arrived, so the uploads overlap the encoding of the jobs
 * already on the device; with the persistent kernel, or when a cube is in
 * pageable memory, the copies precede the batch.  The captured graph is
 * keyed by the host pointers too.  host_src may be NULL (no copies).
 * Synchronous. */
xv_status xv_encode_batch_from_host(xv_ctx* ctx, const xv_job* jobs, const void* const* host_src, int njobs,
                                    xv_result* results, void* stream);

/* SSIM per real band (the paper's Sec. 2.3 quality metric, Wang et al.
 * 2004): band b against its reconstruction x^ = min + q (max - min)/1023
 * (group b/3, channel b%3 of recon), per frame over every 11 x 11 window
 * inside the H x W region with Gaussian weights (sigma 1.5, normalised),
 * local means mu, variances sum w (x - mu)^2 and covariance,
 * SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
 * C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = max - min of the band; windows with a
 * non-finite original sample are skipped; the band's value is the mean over
 * its frames' windows (1 for a constant band, NaN when no window fits).
 * Evaluated in FP32 on (x - min)/L (the index is invariant to it).
 * ssim_band: HOST [bands] or NULL; ssim_mean: HOST, the mean over bands, or
 * NULL.  Synchronous. */
xv_status xv_ssim(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                  const uint16_t* recon, int Hp, int Wp, const double* minmax, double* ssim_band,
                  double* ssim_mean, void* stream);

/* Mean spectral angle (the paper's Sec. 2.3, Kruse et al. 1993), radians:
 * per pixel (t, y, x) of the valid region, the angle between the original
 * spectrum s = (x_b) and the reconstructed one s^ = (x^_b) over all bands,
 * atan2(|s ^ s^|, <s, s^>) with |s ^ s^|^2 = sum over i < j of
 * (s_i s^_j - s_j s^_i)^2 (= acos of the normalised dot product, accurate
 * for small angles); pixels with a non-finite sample or a zero spectrum are
 * skipped.  sa, npix: HOST.  Synchronous. */
xv_status xv_sa(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                const uint16_t* recon, int Hp, int Wp, const double* minmax, double* sa, int64_t* npix,
                void* stream);

/* ------------------------------------------------------ PCA over bands */

/* The paper's optional transform before packing (Sec. 2.1: keep the first
 * nPC principal components of a video's bands; Sec. 3 compresses them as
 * bands, later components at lower quality or not at all).  Every pixel
 * (t, y, x) whose bands are all finite is a sample: mean = the sample mean,
 * covariance = (1/n) sum (x - mean)(x - mean)^T (in double), eigenvectors by
 * cyclic Jacobi rotations in double on the host.  mean: HOST [bands];
 * components: HOST [bands][bands], rows = eigenvectors in order of
 * decreasing eigenvalue (ties: lower index first), each signed so that its
 * first entry of largest magnitude is positive; variance: HOST [bands], the
 * eigenvalues.  XV_EINVAL when no pixel has all bands finite.  Synchronous. */
xv_status xv_pca_fit(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                     double* mean, double* components, double* variance, void* stream);

/* z_k = sum_b components[k][b] (x_b - mean_b) for k < npc, in FP32: src
 * device [bands][T][H][W]; mean, components: HOST (as xv_pca_fit returns
 * them, the first npc rows used); dst: device float32 [npc][T][H][W] (a pixel
 * with a non-finite band gives non-finite components). */
xv_status xv_pca_project(xv_ctx* ctx, const void* src, xv_dtype dtype, int bands, int T, int H, int W,
                         const double* mean, const double* components, int npc, float* dst, void* stream);

/* The inverse: x_b = mean_b + sum_{k < npc} components[k][b] z_k, FP32.
 * z: device float32 [npc][T][H][W]; dst: device float32 [bands][T][H][W]. */
xv_status xv_pca_inverse(xv_ctx* ctx, const float* z, int npc, int bands, int T, int H, int W,
                         const double* mean, const double* components, float* dst, void* stream);

/* ------------------------------------- options: intra frame, deblocking */

/* Frame 0 of G groups with intra prediction (the XV_INTRA option).  Per CU
 * (size N = ctu), in raster order: the 4N + 1 reference samples of each
 * channel -- p[-1][y] and p[x][-1] for 0 <= x, y < 2N and the corner -- from
 * the reconstruction of the CUs coded before it (left, top-left, top,
 * top-right; the below-left never; nothing outside the plane), unavailable
 * samples substituted as in H.265 (in the scan from p[-1][2N-1] up to the
 * corner and along the top row, a missing first sample takes the first
 * available one, every other missing sample its predecessor; none available:
 * all 2^(B-1)); the 35 predictions of H.265 (0 planar, 1 DC, 2..34 angular
 * with the standard's angles and two-tap interpolation; no reference
 * smoothing, no boundary filters) of channel 0, the one with the least SATD
 * (sum over 8 x 8 blocks of (sum |Hadamard| + 2) >> 2; ties to the lower
 * mode) predicts all three channels; then the CU is transformed, quantised
 * and reconstructed as in xv_transform_quant_recon.  Rate proxy per CU: 2 +
 * 6 (mode) + the coded TUs.  The GPU runs the CUs as a wavefront (CU (r, c)
 * after (r, c - 1) and (r - 1, c + 1)), (nx - 1) + 2 (ny - 1) + 1 launches.
 * cur/recon/levels: as in xv_transform_quant_recon (levels may be NULL).
 * mode_mv: int16 [G][nCU][2] at + g * pu_gstride * 2: (mode, 0) per CU.
 * tu_log2 may be NULL; bits: group g's total is ADDED to bits[g * bits_gstride]. */
xv_status xv_intra_frame(xv_ctx* ctx, const uint16_t* cur, int G, int64_t plane_gstride, int Hp, int Wp,
                         const xv_params* p, int64_t pu_gstride, uint16_t* recon, int16_t* levels,
                         uint8_t* tu_log2, int16_t* mode_mv, uint64_t* bits, int64_t bits_gstride, void* stream);

/* Deblocks G reconstructed frames in place (the XV_DEBLOCK option): the H.265
 * luma deblocking filter on each of the three channels.  Edges: the lines of
 * the 8 x 8 grid (not the plane's border) where a CU begins or a TU of the CU
 * holding the edge's first sample after it.  Per 4-sample segment, boundary
 * strength 2 when intra != 0, else 1 when the TU on either side has a
 * non-zero level in any channel or the two CUs' vectors differ by >= 4
 * quarter samples in x or y, else 0 (no filtering); beta = beta'(Clip3(0,
 * 51, qp)) 2^(B-8), tC = tC'(Clip3(0, 53, qp + 2 (bs - 1))) 2^(B-8); the
 * standard's decisions (d < beta; strong when both test lines pass, else
 * weak with |Delta| < 10 tC) and filters.  Every vertical edge of the frame
 * first, then every horizontal edge on that result.  recon: as in
 * xv_transform_quant_recon (read and written); tu_log2: uint8 [G][nCU] and
 * levels (plane layout) of the frame; mv: int16 [G][nCU][2] (read only when
 * intra == 0).  All at the given group strides. */
xv_status xv_deblock_frame(xv_ctx* ctx, uint16_t* recon, int G, int64_t plane_gstride, int Hp, int Wp,
                           const xv_params* p, int64_t pu_gstride, const uint8_t* tu_log2, const int16_t* levels,
                           const int16_t* mv, int intra, void* stream);

/* ------------------------------------------------------ decoder */

/* The decoder (the paper's video2xarray step, Sec. 2.1, below the codec): a
 * frame is rebuilt from its coded data exactly as the encoder reconstructed
 * it.  Per CU: the encoder's prediction (ref == NULL, frame 0: flat 512;
 * else the CU's quarter-sample vector on all three channels of the previous
 * reconstruction, as at xv_transform_quant_recon), then per TU of the CU's
 * size the dequantised levels, the inverse transform and
 * recon = clip(pred + r, 0, 1023).  The rate proxy of
 * xv_transform_quant_recon is recomputed from the levels and vectors, so
 * decoding an encoder's output reproduces its recon and bits bit for bit.
 * Decoding one frame for G groups; layouts as xv_transform_quant_recon:
 * levels: int16 plane layout (group g at + g * plane_gstride, [3][Hp][Wp]);
 * ref/recon: uint16 the same; mv: int16 [G][nCU][2] at + g * pu_gstride * 2
 * (ignored when ref == NULL); tu_log2: uint8 [G][nCU] at + g * pu_gstride
 * (values outside 2..log2 ctu are clamped into it); bits: uint64, group g's
 * frame total is ADDED to bits[g * bits_gstride] (zero it first).  Only
 * p->ctu, p->qp and p->flags are used.  With the encoder's options: XV_INTRA
 * decodes a frame with ref == NULL as xv_intra_frame coded it (CUs as a
 * wavefront, each predicted from its decoded neighbours with the mode in
 * mv[cu][0]; mv is then required), XV_DEBLOCK deblocks the decoded frame in
 * place as xv_deblock_frame does (call the frames in order: a frame is the
 * next one's reference only once it is deblocked). */
xv_status xv_decode_frame(xv_ctx* ctx, const int16_t* levels, const uint16_t* ref, const int16_t* mv,
                          const uint8_t* tu_log2, int G, int64_t plane_gstride, int Hp, int Wp,
                          const xv_params* p, int64_t pu_gstride, uint16_t* recon, uint64_t* bits,
                          int64_t bits_gstride, void* stream);

/* One coded cube for xv_decode_batch (device pointers). */
typedef struct {
    xv_params p;            /* ctu, qp, and search_range: every vector lies within
                               +-(4 search_range + 3) quarter samples (the frame
                               dependency is scheduled from it) */
    int G, T, Hp, Wp;       /* planes: G groups of T frames of [3][Hp][Wp] */
    const int16_t* levels;  /* [G][T][3][Hp][Wp] */
    const int16_t* mv;      /* [G][T][nCU][2] quarter samples (frame 0 ignored) */
    const uint8_t* tu_log2; /* [G][T][nCU] */
    uint16_t* recon;        /* [G][T][3][Hp][Wp], written */
    uint64_t* bits;         /* [G][T] rate proxy per frame, written; or NULL */
    /* the reconstruction in the cube's units (optional, as xv_unpack) */
    int bands, H, W;        /* 1 <= bands <= 3G, H <= Hp, W <= Wp */
    const double* minmax;   /* [bands][2] */
    float* dst;             /* [bands][T][H][W]; NULL: not written */
} xv_djob;

/* Decodes whole cubes in ONE persistent launch per CTU size, scheduled like
 * xv_encode_batch (an item runs once the previous frame's reconstruction rows
 * its vectors can reach are complete); each job's recon equals
 * xv_decode_frame applied frame by frame.  total_bits: HOST [njobs] (the
 * jobs' rate proxies) or NULL.  Synchronous.  XV_ETIMEOUT if a bounded
 * device wait ran out of time; XV_EINVAL on a malformed job (njobs 1..255,
 * 16-byte-aligned levels/recon). */
xv_status xv_decode_batch(xv_ctx* ctx, const xv_djob* jobs, int njobs, uint64_t* total_bits, void* stream);

/* The reconstruction in the cube's units (the inverse of xv_quantize_pack):
 * band b from group b/3, channel b%3 of recon [G][T][3][Hp][Wp] over the valid
 * H x W region, x^ = min + q (max - min)/1023 evaluated in double (multiply,
 * then add) and rounded to float32.  minmax: device [bands][2]; dst: device
 * float32 [bands][T][H][W]. */
xv_status xv_unpack(xv_ctx* ctx, const uint16_t* recon, int bands, int T, int H, int W, int Hp, int Wp,
                    const double* minmax, float* dst, void* stream);

/* ------------------------------------------------------ serving */

/* A compression request for the serving loop.  Unlike xv_job, the cube is in
 * HOST memory (pinned memory makes the upload asynchronous); the library
 * allocates the device buffers itself, under the context's memory budget,
 * and frees them when the request completes.  Every host buffer must stay
 * valid until xv_serve_poll reports the request done. */
typedef struct {
    const void* src;       /* HOST [bands][T][H][W] float32 or uint16 */
    xv_dtype dtype;
    int bands, T, H, W;
    xv_params p;
    uint16_t* recon_out;   /* HOST [G][T][3][Hp][Wp] reconstruction, or NULL */
    int16_t* mv_out;       /* HOST [G][T][nPU][2] motion vectors, or NULL */
} xv_request;

/* Starts the serving loop on the context's device (a library thread).
 * Requests are admitted in submission order while fewer than `max_slots`
 * (1..255) are resident and their device buffers fit the memory budget given
 * to xv_create (0 = no limit); admission uploads and quantises the cube on a
 * copy stream, overlapping the running work.  Each tick advances every
 * resident request by up to `frames_per_tick` frames in one persistent launch
 * (the xv_encode_batch kernel over frame windows), so requests that arrive
 * while others run join at the next tick: continuous batching at frame
 * granularity.  Results are bit-identical to xv_encode_cube.  One serving
 * loop per context; the context's other calls may be used meanwhile. */
xv_status xv_serve_start(xv_ctx* ctx, int max_slots, int frames_per_tick);
/* Queues a request; never blocks.  XV_EBUSY when 65536 requests are queued,
 * XV_EINVAL on a malformed request.  *ticket identifies it. */
xv_status xv_serve_submit(xv_ctx* ctx, const xv_request* req, uint64_t* ticket);
/* Non-blocking.  *done = 1 once the request finished (result filled,
 * including result->status and result->latency_s, the time from submission
 * to completion); the ticket is then released (later polls: XV_ENOTFOUND).
 * When the request failed (result->status != XV_OK), xv_last_error on the
 * polling thread returns its message. */
xv_status xv_serve_poll(xv_ctx* ctx, uint64_t ticket, xv_result* result, int* done);
/* Cancels a queued or resident request; it completes with XV_ECANCELLED at
 * the next tick boundary (unless it finished first). */
xv_status xv_serve_cancel(xv_ctx* ctx, uint64_t ticket);
/* Ticks run, persistent-kernel milliseconds, the largest number of resident
 * requests and the device bytes requests hold now. */
xv_status xv_serve_stats(xv_ctx* ctx, uint64_t* ticks, double* kernel_ms, int* peak_resident, size_t* bytes_in_use);
/* Stops the loop: queued and resident requests are cancelled, the thread is
 * joined, all serving memory is freed.  Unpolled results are discarded. */
xv_status xv_serve_stop(xv_ctx* ctx);

/* ------------------------------------------------------ measurement */

/* Device time of the encode section of the last xv_encode_batch on this
 * context: the persistent kernel launches, or in the per-frame mode the jobs'
 * per-frame chains from their fork to their join (CUDA events recorded on the
 * call's stream around them), in milliseconds.  Host only. */
xv_status xv_last_batch_kernel_ms(const xv_ctx* ctx, double* ms);
/* xv_encode_batch runs a batch as one CUDA graph: captured on the first call
 * with a given set of jobs (shapes, parameters and buffer pointers) and the
 * autotuned block size or mode, replayed while the same batch is submitted
 * again.
 * `enable` = 0 launches the same kernels directly instead.  Host only. */
xv_status xv_set_batch_graphs(xv_ctx* ctx, int enable);
/* Graphs captured and graph launches so far on this context.  Host only. */
xv_status xv_batch_graph_stats(const xv_ctx* ctx, uint64_t* captures, uint64_t* launches);
/* Threads per block of the last xv_encode_batch persistent launch (the
 * autotuner's choice for that batch shape), or 1 when the autotuner chose the
 * per-frame mode (see xv_encode_batch).  Host only. */
xv_status xv_last_batch_block_size(const xv_ctx* ctx, int* block_size);
/* Integer-search work of the last xv_encode_batch on this context.
 * `full_candidates`: the candidates of the integer full search defined at
 * xv_motion_search, (2R + 1)^2 per PU of every frame after the first.
 * `exact_candidates`: those whose SAD the kernels computed exactly (8 per
 * 8-wide unit of vectors, 1 per single last-column unit); the others were
 * excluded by the sub-block sum bound and cannot be the minimum.  Either
 * pointer may be NULL.  Host only. */
xv_status xv_last_batch_search_stats(const xv_ctx* ctx, uint64_t* exact_candidates, uint64_t* full_candidates);
/* The configuration the last xv_encode_batch ran for its CTU class `ctu`
 * (8, 16, 32, 64): *block_size = the persistent kernel's block size, or 1
 * for the per-frame mode (0: the class had no work); *blocks_per_sm = the
 * cap on resident blocks per SM (0: as many as fit), may be NULL.  Host
 * only. */
xv_status xv_last_batch_config(const xv_ctx* ctx, int ctu, int* block_size, int* blocks_per_sm);
/* The autotuner's timings of its last run on this context: one entry per
 * candidate, "ctu<C> nt<B> per<P> <ms>;" for a class's persistent
 * configuration and "frames <ms>;" for the per-frame mode (median of three
 * replays of the captured candidate); "" before any tuning.  The string is
 * owned by the context.  Host only. */
const char* xv_last_tune_log(const xv_ctx* ctx);
/* Number of kernels this context has launched so far.  Host only. */
uint64_t xv_ctx_launches(const xv_ctx* ctx);

/* ------------------------------------------------------ measurement */

/* Device microbenchmark of an instruction sequence that the benchmark's
 * roofline fractions are quoted against (not a step of the method): the
 * rate, over the whole device, of
 *   kind 0: abs-diff-accumulates as one integer sad instruction each,
 *   kind 1: abs-diff-accumulates on the FP32 pipe (subtract, add |.|),
 *   kind 2: the mix of two kind-0 per kind-1 (both pipes at once),
 *   kind 3: 32-bit integer multiply-adds (the transform's operation).
 * Every SM runs at its thread limit; best of three timed runs after one
 * warm-up, on the legacy default stream.  *rate: operations per second;
 * *ms: that run's duration (may be NULL).  Synchronous.  XV_EINVAL for a
 * kind outside 0..3. */
xv_status xv_measure_peak(xv_ctx* ctx, int kind, double* rate, double* ms);

/* ------------------------------------------------------ test hooks */

/* Spin budget (SM clock cycles, default 4e9, about 2 s) of each dependency
 * wait in xv_encode_batch.  Host only. */
xv_status xv_debug_set_wait_budget(xv_ctx* ctx, long long cycles);
/* Run xv_encode_batch with this block size (128, 192, 256 or 512, plus
 * 1024 x a cap on resident blocks per SM, 1..32, if wanted), or 1 for its
 * per-frame mode, instead of the autotuner's choice, captured and replayed
 * as CUDA graphs exactly as a tuned choice is; 0 restores the autotuner.
 * Host only. */
xv_status xv_debug_force_block_size(xv_ctx* ctx, int block_size);
/* Bound (mbarrier polls, default 2^24; 0 restores it) of the per-frame
 * search's wait for its window copy (the window comes by TMA where it lies
 * inside the plane); a negative value turns the TMA copies off (every window
 * by the threads' own 16-byte loads, for comparison).  A copy that does not
 * complete within the bound makes xv_encode_cube / xv_encode_batch
 * (per-frame mode) return XV_ETIMEOUT without any fault; the context stays
 * usable.  Host only. */
xv_status xv_debug_set_window_wait(xv_ctx* ctx, long long polls);
/* Make one dependency counter of xv_encode_batch impossible to complete: the
 * CTU row `row` of the first job, indexed over its [G][T][rows] counters, is
 * then never queued, a block waiting for it runs out of its budget, and the
 * batch returns XV_ETIMEOUT without any fault; -1 disables.  Host only. */
xv_status xv_debug_stall_row(xv_ctx* ctx, long long row);

#ifdef __cplusplus
}
#endif
#endif /* XV_H */
