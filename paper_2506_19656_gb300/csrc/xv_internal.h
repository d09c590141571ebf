// xv_internal.h -- host-side internals of libxv shared by the .cu files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/xv.h"

namespace xvh {

// Per-band quantiser constants computed on the device from min/max.
struct BandQ {
    double lo, hi, s, delta;  // s = 1023/(hi-lo) (0 if hi <= lo); delta = (hi-lo)/1023
    float lo_f, s_f;          // float copies for the exact fast path
    int fast_ok;              // lo is a float value and s is in float range
    int pad;
};

// Device scratch regions owned by a context (grown on demand).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

void set_error(const char* fmt, ...);
// The calling thread's last error message.
const char* last_error_text();
xv_status cuda_fail(cudaError_t e, const char* what);

// ---- launchers (stream = cudaStream_t)
cudaError_t launch_minmax(const void* src, xv_dtype dt, int bands, int64_t n_per_band, unsigned* enc,
                          double* minmax, BandQ* bq, cudaStream_t st);
cudaError_t launch_bandq(const double* minmax, int bands, BandQ* bq, cudaStream_t st);
cudaError_t launch_quantize_pack(const void* src, xv_dtype dt, int bands, int T, int H, int W, int Hp, int Wp,
                                 const BandQ* bq, uint16_t* planes, cudaStream_t st);

// A tensor map (CUtensorMap, 128 bytes) for the TMA loads of the search
// window over the G groups' channel-0 planes of one frame (tma.cu);
// valid = 0: not usable here (the search loads the window itself).
struct alignas(64) WindowMap {
    unsigned char bytes[128];
    int valid;
    long long polls;  // the bound of the wait for the copy (mbarrier polls)
};
bool window_map_usable(int ctu, int R);
bool encode_window_map(WindowMap* m, const uint16_t* plane0, int Wp, int Hp, int64_t gstride, int G, int ctu, int R);

// exact: when not null, the integer-search candidates evaluated exactly are added to *exact.
// wmap (valid) and err: the window by TMA, a copy that does not complete
// within the wait bound setting *err to XV_ETIMEOUT.
cudaError_t launch_me_frame(const uint16_t* cur, const uint16_t* ref, int G, int64_t gstride, int Hp, int Wp,
                            const xv_params* p, int16_t* mv, uint32_t* cost, int16_t* mv_int,
                            uint32_t* cost_int, int64_t pu_gstride, cudaStream_t st,
                            unsigned long long* exact = nullptr, const WindowMap* wmap = nullptr, int* err = nullptr);
// Microbenchmarks of the roofline's instruction sequences (k_peak.cu): kind
// 0..3 (see the file); sink receives at most one word per block.
int peak_chains();
cudaError_t launch_peak(int kind, const uint32_t* in, int iters, uint32_t* sink, int* threads_out,
                        cudaStream_t st);
// PCA over bands (k_pca.cu).
int pca_fit_blocks(int64_t npix);
cudaError_t launch_pca_sums(const void* src, xv_dtype dt, int bands, int64_t npix, double* part, int nblk,
                            cudaStream_t st);
cudaError_t launch_pca_cov(const void* src, xv_dtype dt, int bands, int64_t npix, const double* mean, double* part,
                           int nblk, cudaStream_t st);
cudaError_t launch_pca_project(const void* src, xv_dtype dt, int bands, int npc, int64_t npix, const double* mean,
                               const double* comps, float* dst, cudaStream_t st);
cudaError_t launch_pca_inverse(const float* z, int npc, int bands, int64_t npix, const double* mean, const double* comps,
                               float* dst, cudaStream_t st);
void pca_eigen(int n, const double* a, double* vals, double* vecs);
// SSIM / spectral-angle partial sums (k_metrics.cu).
struct MetricPart {
    double sum;
    unsigned long long n;
};
int ssim_blocks_per_band(int T, int H, int W);
int sa_blocks(int64_t npix);
cudaError_t launch_ssim(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* recon, int Hp,
                        int Wp, const BandQ* bq, MetricPart* part, int nblk, MetricPart* out, cudaStream_t st);
cudaError_t launch_sa(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* recon, int Hp,
                      int Wp, const BandQ* bq, MetricPart* part, int nblk, MetricPart* out, cudaStream_t st);
cudaError_t launch_dec_frame(const int16_t* levels, const uint16_t* ref, const int16_t* mv, const uint8_t* tu_log2,
                             int G, int64_t gstride, int Hp, int Wp, const xv_params* p, int64_t pu_gstride,
                             uint16_t* recon, uint64_t* bits, int64_t bits_gstride, cudaStream_t st);
cudaError_t launch_unpack(const uint16_t* recon, int bands, int T, int H, int W, int Hp, int Wp, const double* minmax,
                          float* dst, cudaStream_t st);
size_t decode_smem_bytes(int ctu);
cudaError_t launch_tqr_frame(const uint16_t* cur, const uint16_t* ref, const int16_t* mv, int G, int64_t gstride,
                             int Hp, int Wp, const xv_params* p, int64_t pu_gstride, uint16_t* recon,
                             int16_t* levels, uint8_t* tu_log2, uint64_t* bits, int64_t bits_gstride,
                             cudaStream_t st);

// PSNR partial sums: per band, `nblk` partials of (sse double, sse10, count).
struct PsnrPart {
    double sse;
    unsigned long long sse10;
    unsigned long long count;
    double pad;
};
int psnr_blocks_per_band(int64_t samples_per_band, int bands);
cudaError_t launch_psnr(const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* planes,
                        const uint16_t* recon, int Hp, int Wp, const BandQ* bq, PsnrPart* part, int nblk,
                        PsnrPart* out, cudaStream_t st);

}  // namespace xvh

namespace xvh {

// One cube of a batch, as the persistent kernel sees it.
struct JobDev {
    const uint16_t* planes;  // [G][T][3][Hp][Wp]
    uint16_t* recon;
    int16_t* mv;             // [G][T][nPU][2] or null
    uint32_t* cost;          // [G][T][nPU] or null
    int16_t* levels;         // plane layout or null
    uint8_t* tu;             // [G][T][nPU] or null
    uint64_t* bits;          // [G][T]
    unsigned* rowdone;       // [G][T][ny]: finished PUs per CTU row
    unsigned* depcnt;        // [G][T][ny]: finished rows of the previous frame a row reads
    int64_t lf8, lmv;
    int G, T, Hp, Wp, ctu, R, qp;
    unsigned tu_mask;
    int nx, ny;
    int64_t qfirst;          // queue slot of this job's first window item
    int tb, te;              // frames [tb, te) are encoded by this launch (frame tb-1 is complete)
};

// One CTU class of a batch, as the prologue sees it.
struct ClassDev {
    int64_t qoff;            // first queue slot of the class
    unsigned total;          // items of the class
    unsigned nfirst;         // items of the jobs' first window frames (queued by the prologue)
};

// Ready-queue control block (device).
struct BatchCtl {
    unsigned head;         // next queue position to take
    unsigned tail;         // next queue position to fill
    unsigned total;        // items in the launch (every item is queued once)
    int err;               // 0, or an xv_status (XV_ETIMEOUT) set by a block
    long long budget;      // spin budget per wait, in SM clock cycles
    long long stall_row;   // test hook: this dependency counter never completes (-1: none)
    unsigned long long exact_cand;  // integer-search candidates whose SAD was computed exactly
};

// Item key: job (8 bits) | group (8) | frame (16) | PU (32).
constexpr uint64_t kEmptyItem = ~0ull;
inline uint64_t make_item(int job, int g, int t, int pu) {
    return ((uint64_t)job << 56) | ((uint64_t)g << 48) | ((uint64_t)t << 32) | (uint32_t)pu;
}

size_t persist_smem_bytes(int ctu, int R, bool has_me);
// Resets each job's counters and bits over its frame window, fills the
// queues (the window's first-frame items, then empty slots) and the control
// blocks.
cudaError_t launch_batch_prologue(const JobDev* jobs, int njobs, const ClassDev* cls, uint64_t* queue,
                                  BatchCtl* ctl, long long budget, long long stall_row, cudaStream_t st);
// min/max (unless fixed) and the per-band quantiser constants; `enc` is
// 2 * bands words of scratch.
cudaError_t launch_prepare_bands(const void* src, xv_dtype dt, int bands, int64_t n_per_band, double* minmax,
                                 int fixed, unsigned* enc, BandQ* bq, cudaStream_t st);
// totals[j] = sum of job j's per-frame bits.
cudaError_t launch_bits_totals(const JobDev* jobs, int njobs, unsigned long long* totals, cudaStream_t st);
// Block sizes the persistent kernel is built for (the autotuner picks one).
constexpr int kPersistBlockSizes[4] = {128, 192, 256, 512};
// Frame-0 intra coding of G groups: a wavefront of launches (*launches counts them).
cudaError_t launch_intra_frame(const uint16_t* cur, int G, int64_t gstride, int Hp, int Wp, const xv_params* p,
                               int16_t* mv, int64_t pu_gstride, uint16_t* recon, int16_t* levels, uint8_t* tu_log2,
                               uint64_t* bits, int64_t bits_gstride, cudaStream_t st, uint64_t* launches);
// Decoding of frame 0 of G groups with intra prediction (modes in mode_mv[cu][0]).
cudaError_t launch_intra_decode_frame(const int16_t* levels, int G, int64_t gstride, int Hp, int Wp, int ctu, int qp,
                                      const int16_t* mode_mv, int64_t pu_gstride, const uint8_t* tu_log2,
                                      uint16_t* recon, uint64_t* bits, int64_t bits_gstride, cudaStream_t st,
                                      uint64_t* launches);
// In-place deblocking of G reconstructed frames; cbf: G (Hp / 4) (Wp / 4) bytes of scratch.
cudaError_t launch_deblock_frame(uint16_t* recon, int G, int64_t gstride, int Hp, int Wp, int ctu, int qp,
                                 const uint8_t* tu_log2, int64_t pu_gstride, const int16_t* levels,
                                 const int16_t* mv, int intra, uint8_t* cbf, cudaStream_t st, uint64_t* launches);
// decode: the decoding instantiation (the jobs' levels, vectors and TU sizes
// are inputs, recon and bits outputs) instead of the encoder.
cudaError_t launch_persist(int ctu, int nt, bool decode, const JobDev* jobs, uint64_t* queue, BatchCtl* ctl,
                           size_t smem, int grid, cudaStream_t st);
// Grid of a persistent launch: every SM times the resident blocks per SM
// (at most per_cap of them when per_cap > 0).
int persist_grid(int ctu, int nt, size_t smem, bool decode, int per_cap = 0);
// Resident blocks per SM of a persistent kernel configuration.
inline int persist_blocks_per_sm(int ctu, int nt, size_t smem, bool decode) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return persist_grid(ctu, nt, smem, decode) / (sms > 0 ? sms : 1);
}

}  // namespace xvh

namespace xvh {

// Serving (csrc/xv_serve.cu).
struct ServeState;
// block / per_cap: the persistent kernel's block size and resident-block cap
// per SM for each CTU class (8, 16, 32, 64).
ServeState* serve_create(int device, int max_slots, int frames_per_tick, size_t budget, long long wait_budget,
                         const int block[4], const int per_cap[4], xv_status* st);
void serve_destroy(ServeState* s);
xv_status serve_submit(ServeState* s, const xv_request* r, uint64_t* ticket);
xv_status serve_poll(ServeState* s, uint64_t ticket, xv_result* res, int* done);
xv_status serve_cancel(ServeState* s, uint64_t ticket);
void serve_stats(ServeState* s, uint64_t* ticks, double* kernel_ms, int* peak_active, size_t* bytes_in_use);

}  // namespace xvh
