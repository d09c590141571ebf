// xv_api.cu -- the C ABI of include/xv.h: context, argument checks, the plain
// (per-frame) and batched (persistent) cube paths, and PSNR finalisation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

using xvh::BandQ;
using xvh::DevBuf;

struct xv_ctx {
    int device = 0;
    size_t budget = 0;  // 0 = unlimited
    size_t held = 0;
    // scratch of the single-cube calls
    DevBuf mm_enc, bandq, psnr_part, psnr_out, tmp_mv, tmp_bits, tmp_minmax, met_part, met_out, pca_part, tmp_cbf;
    // scratch of the batched path
    DevBuf b_jobs, b_items, b_rowdone, b_depcnt, b_ctl, b_bits, b_bandq, b_minmax;
    long long wait_budget = 4000000000LL;  // cycles per dependency wait (about 2 s)
    long long stall_row = -1;              // test hook (xv_debug_stall_row)
    uint64_t launches = 0;                 // kernels launched by this context
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the persistent launches
    double batch_ms = 0.0;
    int batch_nt = 0;                        // block size of the last persistent launch
    uint64_t batch_exact = 0, batch_full = 0;  // integer-search candidates: evaluated exactly / defined
    std::map<std::string, int> tuned_nt;     // autotuner: batch shape -> block size
    int force_nt = 0;                        // test hook (xv_debug_force_block_size)
    // batched path: buffers, work stream and the captured graph
    DevBuf b_cls, b_part, b_out, b_totals;
    void* h_stage = nullptr;                 // pinned host copy of a batch's results
    size_t h_stage_bytes = 0;
    cudaStream_t work = nullptr;             // batches run here (capturable, ordered after the caller's stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // setup, persistent kernels, results
    std::string graph_key;
    int use_graph = 1;
    uint64_t graph_launches = 0, graph_captures = 0;
    // the batched path's second execution mode: the jobs as per-frame chains
    // on side streams (vectors of jobs without an mv buffer, exact-candidate count)
    cudaStream_t side[16] = {};
    cudaEvent_t side_ev[16] = {};
    cudaEvent_t fork_ev = nullptr;
    // xv_encode_batch_from_host: the cubes' uploads on their own stream, one
    // completion event per job
    cudaStream_t up_st = nullptr;
    cudaEvent_t up_join = nullptr;
    std::vector<cudaEvent_t> up_ev;
    DevBuf b_mv, b_exact, b_mm_enc;
    DevBuf peak_buf;                         // xv_measure_peak's input and sink
    DevBuf dev_err;                          // status word the per-frame search sets on a copy timeout
    long long tma_polls = 1ll << 24;         // bound of the search window copy's wait (test hook)
    bool tma_off = false;                    // the search loads every window itself (test hook)
    int batch_cfg[4] = {0, 0, 0, 0};         // configuration code of each CTU class in the last batch
    int class_tuned[4] = {0, 0, 0, 0};       // the autotuner's latest persistent choice per CTU class
    std::string tune_log;                    // the autotuner's last timings
    xvh::ServeState* serve = nullptr;
};

// Block size value that selects the batched path's per-frame mode.
constexpr int kFramesMode = 1;
// A persistent-kernel configuration of one CTU class: block size + 1024 x
// the cap on resident blocks per SM (0: as many as fit).
constexpr int cfg_code(int nt, int per_cap) { return nt + 1024 * per_cap; }
constexpr int cfg_nt(int code) { return code == kFramesMode ? kFramesMode : code % 1024; }
constexpr int cfg_per(int code) { return code == kFramesMode ? 0 : code / 1024; }
constexpr int kSideStreams = 16;

namespace xvh {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

xv_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return XV_ECUDA;
}

const char* last_error_text() { return g_err.c_str(); }

}  // namespace xvh

using xvh::cuda_fail;
using xvh::set_error;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

xv_status ensure(xv_ctx* c, DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (b.bytes >= bytes) return XV_OK;
    size_t nb = (bytes + 255) / 256 * 256;
    if (c->budget && c->held - b.bytes + nb > c->budget) {
        set_error("device scratch of %zu bytes exceeds the context budget (%zu of %zu held)", nb, c->held,
                  c->budget);
        return XV_EBUDGET;
    }
    if (b.ptr) {
        cudaDeviceSynchronize();
        cudaFree(b.ptr);
        c->held -= b.bytes;
        b = DevBuf{};
    }
    cudaError_t e = cudaMalloc(&b.ptr, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu): %s", nb, cudaGetErrorString(e));
        return XV_ENOMEM;
    }
    b.bytes = nb;
    c->held += nb;
    return XV_OK;
}

void release(xv_ctx* c, DevBuf& b) {
    if (b.ptr) {
        cudaFree(b.ptr);
        c->held -= b.bytes;
    }
    b = DevBuf{};
}

bool valid_params(const xv_params* p) {
    if (!p) { set_error("params is NULL"); return false; }
    if (p->bit_depth != 10) { set_error("bit_depth %d: only 10 is supported", p->bit_depth); return false; }
    if (p->ctu != 8 && p->ctu != 16 && p->ctu != 32 && p->ctu != 64) {
        set_error("ctu %d: must be 8, 16, 32 or 64", p->ctu);
        return false;
    }
    if (p->search_range < 1 || p->search_range > 64) {
        set_error("search_range %d: must be in 1..64", p->search_range);
        return false;
    }
    if (p->tu_mask & ~0x3cu) { set_error("tu_mask 0x%x: only bits 2..5 (TU 4..32) may be set", p->tu_mask); return false; }
    bool any = false;
    for (int k = 2; k <= 5; ++k)
        if ((p->tu_mask & (1u << k)) && (1 << k) <= p->ctu) any = true;
    if (!any) { set_error("tu_mask 0x%x allows no TU size <= ctu %d", p->tu_mask, p->ctu); return false; }
    if (p->qp < -12 || p->qp > 51) { set_error("qp %d: must be in [-12, 51]", p->qp); return false; }
    if (p->flags & ~(XV_INTRA | XV_DEBLOCK)) { set_error("flags 0x%x: only XV_INTRA and XV_DEBLOCK exist", p->flags); return false; }
    if (xvd::me_smem_bytes(p->ctu, p->search_range) > 227 * 1024) {
        set_error("ctu %d with search range %d needs more shared memory than a block has", p->ctu, p->search_range);
        return false;
    }
    return true;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// The intra and deblocking options run on the per-frame path only.
bool no_options(const xv_params* p, const char* where) {
    if (p->flags == 0) return true;
    set_error("%s: the XV_INTRA / XV_DEBLOCK options are supported by xv_encode_cube, xv_decode_frame and the other "
              "per-frame calls only",
              where);
    return false;
}

bool valid_planes(const void* a, const void* b, const void* c, int64_t gstride) {
    if (!aligned16(a) || !aligned16(b) || !aligned16(c) || gstride % 8 != 0) {
        set_error("plane pointers must be 16-byte aligned and the group stride a multiple of 8 samples");
        return false;
    }
    return true;
}

bool valid_frame(int G, int Hp, int Wp, int ctu) {
    if (G < 1 || G > 255) { set_error("G %d: must be in 1..255", G); return false; }
    if (Hp < ctu || Wp < ctu || Hp % ctu || Wp % ctu) {
        set_error("plane %dx%d is not a positive multiple of the CTU size %d", Hp, Wp, ctu);
        return false;
    }
    return true;
}

bool valid_cube(const void* src, xv_dtype dt, int bands, int T, int H, int W) {
    if (!src) { set_error("src is NULL"); return false; }
    if (dt != XV_F32 && dt != XV_U16) { set_error("dtype %d: must be XV_F32 or XV_U16", (int)dt); return false; }
    if (bands < 1 || bands > XV_MAX_BANDS) { set_error("bands %d: must be in 1..%d", bands, XV_MAX_BANDS); return false; }
    if (T < 1 || H < 1 || W < 1) { set_error("cube %dx%dx%d has an empty dimension", T, H, W); return false; }
    if (T > 65535) { set_error("T %d: at most 65535 frames", T); return false; }
    return true;
}

int plane_dim(int n, int ctu) { return (n + ctu - 1) / ctu * ctu; }

// The device status word of the per-frame search (zeroed when created).
xv_status ensure_err_word(xv_ctx* c) {
    if (c->dev_err.ptr) return XV_OK;
    xv_status s = ensure(c, c->dev_err, sizeof(int));
    if (s) return s;
    cudaError_t e = cudaMemset(c->dev_err.ptr, 0, sizeof(int));
    return e == cudaSuccess ? XV_OK : cuda_fail(e, "status word");
}

// The window map of frame t's reference (channel 0 of reconstruction t - 1 of
// every group); invalid (the search loads the window itself) when not usable.
xvh::WindowMap window_map(const xv_ctx* c, const uint16_t* ref_frame, int Wp, int Hp, int64_t gstride, int G,
                          const xv_params& p) {
    xvh::WindowMap m{};
    if (!c->tma_off && xvh::encode_window_map(&m, ref_frame, Wp, Hp, gstride, G, p.ctu, p.search_range))
        m.polls = c->tma_polls;
    return m;
}

// Reads and clears the per-frame search's status word (synchronous).
xv_status take_err_word(xv_ctx* c) {
    if (!c->dev_err.ptr) return XV_OK;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, c->dev_err.ptr, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    if (v == 0) return XV_OK;
    cudaMemset(c->dev_err.ptr, 0, sizeof(int));
    set_error("a search window copy did not complete within its wait bound");
    return (xv_status)v;
}

xv_status check_launch(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(e, what);
    return XV_OK;
}

// Kernels issued by each launcher (for xv_ctx_launches).
constexpr int kLaunchMinmax = 3, kLaunchBandq = 1, kLaunchQuant = 1, kLaunchMe = 1, kLaunchTqr = 1, kLaunchPsnr = 2,
              kLaunchPersist = 1;

// min/max (unless fixed) and the per-band quantiser constants into `bq`;
// `scratch` (2 x bands words) is the reduction's, the context's own when
// null.
xv_status prepare_bands(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, double* minmax,
                        int fixed, BandQ* bq, cudaStream_t st, unsigned* scratch = nullptr) {
    if (fixed) {
        c->launches += kLaunchBandq;
        return check_launch(xvh::launch_bandq(minmax, bands, bq, st), "band constants");
    }
    if (!scratch) {
        xv_status s = ensure(c, c->mm_enc, sizeof(unsigned) * 2 * bands);
        if (s) return s;
        scratch = (unsigned*)c->mm_enc.ptr;
    }
    c->launches += kLaunchMinmax;
    return check_launch(xvh::launch_minmax(src, dt, bands, (int64_t)T * H * W, scratch, minmax, bq, st), "min/max");
}

// PSNR of one cube into `r` (host), from device band constants `bq`.
xv_status psnr_into(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W,
                    const uint16_t* planes, const uint16_t* recon, int Hp, int Wp, const BandQ* bq, double* psnr,
                    double* mse, uint64_t* sse10, double* mean, cudaStream_t st) {
    const int nblk = xvh::psnr_blocks_per_band((int64_t)T * H * W, bands);
    xv_status s = ensure(c, c->psnr_part, sizeof(xvh::PsnrPart) * (size_t)nblk * bands);
    if (s) return s;
    if ((s = ensure(c, c->psnr_out, sizeof(xvh::PsnrPart) * bands))) return s;
    c->launches += kLaunchPsnr;
    s = check_launch(xvh::launch_psnr(src, dt, bands, T, H, W, planes, recon, Hp, Wp, bq,
                                      (xvh::PsnrPart*)c->psnr_part.ptr, nblk, (xvh::PsnrPart*)c->psnr_out.ptr, st),
                     "psnr");
    if (s) return s;
    std::vector<xvh::PsnrPart> out(bands);
    std::vector<BandQ> hq(bands);
    cudaError_t e = cudaMemcpyAsync(out.data(), c->psnr_out.ptr, sizeof(xvh::PsnrPart) * bands,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hq.data(), bq, sizeof(BandQ) * bands, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "psnr read-back");
    double acc = 0.0;
    bool inf = false;
    for (int b = 0; b < bands; ++b) {
        const double cnt = (double)out[b].count;
        const double m = cnt > 0 ? out[b].sse / cnt : 0.0;
        const double peak = hq[b].hi > 0.0 ? hq[b].hi : hq[b].hi - hq[b].lo;
        const double p = m > 0.0 ? 10.0 * std::log10(peak * peak / m) : INFINITY;
        if (psnr) psnr[b] = p;
        if (mse) mse[b] = m;
        if (sse10) sse10[b] = out[b].sse10;
        if (std::isinf(p)) inf = true; else acc += p;
    }
    if (mean) *mean = inf ? INFINITY : acc / bands;
    return XV_OK;
}

xv_status fill_result(const xv_job* j, const uint64_t* bits_dev, int G, xv_result* r, cudaStream_t st) {
    std::vector<uint64_t> hb((size_t)G * j->T);
    cudaError_t e = cudaMemcpyAsync(hb.data(), bits_dev, sizeof(uint64_t) * hb.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "bits read-back");
    uint64_t tot = 0;
    for (uint64_t v : hb) tot += v;
    r->total_bits = tot;
    r->bands = j->bands;
    r->bpppb = (double)tot / ((double)j->H * j->W * j->T * j->bands);
    r->ctu = j->p.ctu;
    r->block_size = 1;  // the per-frame launches
    return XV_OK;
}

bool valid_job(const xv_job* j) {
    if (!j) { set_error("job is NULL"); return false; }
    if (!valid_cube(j->src, j->dtype, j->bands, j->T, j->H, j->W)) return false;
    if (!valid_params(&j->p)) return false;
    if (!j->planes || !j->recon) { set_error("job planes and recon buffers are required"); return false; }
    if (!valid_planes(j->planes, j->recon, j->levels ? (const void*)j->levels : j->planes, 8)) return false;
    if (j->minmax_fixed && !j->minmax) { set_error("minmax_fixed needs a minmax array"); return false; }
    return true;
}

}  // namespace

extern "C" {

const char* xv_last_error(void) { return xvh::g_err.c_str(); }

const char* xv_status_string(xv_status s) {
    switch (s) {
        case XV_OK: return "ok";
        case XV_EINVAL: return "invalid argument";
        case XV_ENOMEM: return "out of device memory";
        case XV_EBUDGET: return "over the memory budget";
        case XV_ETIMEOUT: return "device wait timed out";
        case XV_EBUSY: return "queue full";
        case XV_ECUDA: return "CUDA error";
        case XV_ECANCELLED: return "cancelled";
        case XV_ENOTFOUND: return "not found";
    }
    return "unknown status";
}

xv_status xv_create(xv_ctx** out, int device, size_t budget) {
    if (!out) { set_error("ctx out-pointer is NULL"); return XV_EINVAL; }
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) { set_error("device %d: %d device(s) present", device, n); return XV_EINVAL; }
    xv_ctx* c = new xv_ctx;
    c->device = device;
    c->budget = budget;
    *out = c;
    return XV_OK;
}

void xv_destroy(xv_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->serve) { xvh::serve_destroy(c->serve); c->serve = nullptr; }
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&c->mm_enc, &c->bandq, &c->psnr_part, &c->psnr_out, &c->tmp_mv, &c->tmp_bits, &c->tmp_minmax, &c->tmp_cbf,
                      &c->b_jobs, &c->b_items, &c->b_rowdone, &c->b_depcnt, &c->b_ctl, &c->b_bits, &c->b_bandq,
                      &c->b_minmax, &c->b_cls, &c->b_part, &c->b_out, &c->b_totals, &c->b_mv, &c->b_exact, &c->b_mm_enc,
                      &c->met_part, &c->met_out, &c->pca_part, &c->peak_buf, &c->dev_err};
    for (DevBuf* b : bufs) release(c, *b);
    for (cudaGraphExec_t& gx : c->graph)
        if (gx) cudaGraphExecDestroy(gx);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    for (int k = 0; k < kSideStreams; ++k) {
        if (c->side[k]) cudaStreamDestroy(c->side[k]);
        if (c->side_ev[k]) cudaEventDestroy(c->side_ev[k]);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->up_st) cudaStreamDestroy(c->up_st);
    if (c->up_join) cudaEventDestroy(c->up_join);
    for (cudaEvent_t ev : c->up_ev) cudaEventDestroy(ev);
    if (c->work) cudaStreamDestroy(c->work);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

size_t xv_ctx_bytes(const xv_ctx* c) { return c ? c->held : 0; }

xv_status xv_params_init(xv_params* p, int ctu, int R, unsigned tu_mask, int qp) {
    if (!p) { set_error("params is NULL"); return XV_EINVAL; }
    xv_params q;
    q.bit_depth = 10;
    q.ctu = ctu;
    q.search_range = R;
    q.tu_mask = tu_mask;
    q.qp = qp;
    q.flags = 0u;
    const double lambda = 0.57 * std::pow(2.0, (qp - 12) / 3.0);
    q.lambda_fp8 = std::llround(256.0 * lambda);
    q.lambda_mv_fp16 = std::llround(65536.0 * std::sqrt(lambda));
    if (!valid_params(&q)) return XV_EINVAL;
    *p = q;
    return XV_OK;
}

xv_status xv_plane_geometry(int bands, int H, int W, int ctu, int* G, int* Hp, int* Wp) {
    if (bands < 1 || H < 1 || W < 1 || (ctu != 8 && ctu != 16 && ctu != 32 && ctu != 64)) {
        set_error("bad geometry bands=%d H=%d W=%d ctu=%d", bands, H, W, ctu);
        return XV_EINVAL;
    }
    if (G) *G = (bands + 2) / 3;
    if (Hp) *Hp = plane_dim(H, ctu);
    if (Wp) *Wp = plane_dim(W, ctu);
    return XV_OK;
}

xv_status xv_minmax(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, double* minmax,
                    void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (!minmax) { set_error("minmax is NULL"); return XV_EINVAL; }
    DeviceGuard g(c->device);
    xv_status s = ensure(c, c->bandq, sizeof(BandQ) * bands);
    if (s) return s;
    return prepare_bands(c, src, dt, bands, T, H, W, minmax, 0, (BandQ*)c->bandq.ptr, (cudaStream_t)stream);
}

xv_status xv_quantize_pack(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, int ctu,
                           double* minmax, int fixed, uint16_t* planes, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (ctu != 8 && ctu != 16 && ctu != 32 && ctu != 64) { set_error("ctu %d", ctu); return XV_EINVAL; }
    if (!minmax || !planes) { set_error("minmax and planes are required"); return XV_EINVAL; }
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    xv_status s = ensure(c, c->bandq, sizeof(BandQ) * bands);
    if (s) return s;
    BandQ* bq = (BandQ*)c->bandq.ptr;
    if ((s = prepare_bands(c, src, dt, bands, T, H, W, minmax, fixed, bq, st))) return s;
    c->launches += kLaunchQuant;
    return check_launch(xvh::launch_quantize_pack(src, dt, bands, T, H, W, plane_dim(H, ctu), plane_dim(W, ctu), bq,
                                                  planes, st),
                        "quantize_pack");
}

xv_status xv_motion_search(xv_ctx* c, const uint16_t* cur, const uint16_t* ref, int G, int64_t gstride, int Hp,
                           int Wp, const xv_params* p, int16_t* mv, uint32_t* cost, int16_t* mv_int,
                           uint32_t* cost_int, int64_t pu_gstride, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_params(p) || !valid_frame(G, Hp, Wp, p->ctu)) return XV_EINVAL;
    if (!cur || !ref || !mv) { set_error("cur, ref and mv are required"); return XV_EINVAL; }
    if (!valid_planes(cur, ref, cur, gstride)) return XV_EINVAL;
    DeviceGuard g(c->device);
    c->launches += kLaunchMe;
    return check_launch(xvh::launch_me_frame(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride,
                                             (cudaStream_t)stream),
                        "motion_search");
}

xv_status xv_transform_quant_recon(xv_ctx* c, const uint16_t* cur, const uint16_t* ref, const int16_t* mv, int G,
                                   int64_t gstride, int Hp, int Wp, const xv_params* p, int64_t pu_gstride,
                                   uint16_t* recon, int16_t* levels, uint8_t* tu_log2, uint64_t* bits,
                                   int64_t bits_gstride, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_params(p) || !valid_frame(G, Hp, Wp, p->ctu)) return XV_EINVAL;
    if (!cur || !recon || !bits || (ref && !mv)) { set_error("cur, recon, bits (and mv with ref) are required"); return XV_EINVAL; }
    if (!valid_planes(cur, ref ? ref : cur, recon, gstride)) return XV_EINVAL;
    if (levels && !valid_planes(levels, levels, levels, gstride)) return XV_EINVAL;
    DeviceGuard g(c->device);
    c->launches += kLaunchTqr;
    return check_launch(xvh::launch_tqr_frame(cur, ref, mv, G, gstride, Hp, Wp, p, pu_gstride, recon, levels, tu_log2,
                                              bits, bits_gstride, (cudaStream_t)stream),
                        "transform_quant_recon");
}

xv_status xv_intra_frame(xv_ctx* c, const uint16_t* cur, int G, int64_t gstride, int Hp, int Wp, const xv_params* p,
                         int64_t pu_gstride, uint16_t* recon, int16_t* levels, uint8_t* tu_log2, int16_t* mode_mv,
                         uint64_t* bits, int64_t bits_gstride, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_params(p) || !valid_frame(G, Hp, Wp, p->ctu)) return XV_EINVAL;
    if (!cur || !recon || !bits || !mode_mv) { set_error("cur, recon, mode_mv and bits are required"); return XV_EINVAL; }
    if (!valid_planes(cur, cur, recon, gstride)) return XV_EINVAL;
    if (levels && !valid_planes(levels, levels, levels, gstride)) return XV_EINVAL;
    DeviceGuard g(c->device);
    uint64_t launched = 0;
    xv_status s = check_launch(xvh::launch_intra_frame(cur, G, gstride, Hp, Wp, p, mode_mv, pu_gstride, recon, levels,
                                                       tu_log2, bits, bits_gstride, (cudaStream_t)stream, &launched),
                               "intra frame");
    c->launches += launched;
    return s;
}

// The coded-block scratch of deblocking, G (Hp / 4) (Wp / 4) bytes.
static xv_status deblock_into(xv_ctx* c, uint16_t* recon, int G, int64_t gstride, int Hp, int Wp, const xv_params* p,
                              int64_t pu_gstride, const uint8_t* tu_log2, const int16_t* levels, const int16_t* mv,
                              int intra, cudaStream_t st) {
    xv_status s = ensure(c, c->tmp_cbf, (size_t)G * (Hp / 4) * (Wp / 4));
    if (s) return s;
    uint64_t launched = 0;
    s = check_launch(xvh::launch_deblock_frame(recon, G, gstride, Hp, Wp, p->ctu, p->qp, tu_log2, pu_gstride, levels, mv,
                                               intra, (uint8_t*)c->tmp_cbf.ptr, st, &launched),
                     "deblocking");
    c->launches += launched;
    return s;
}

xv_status xv_deblock_frame(xv_ctx* c, uint16_t* recon, int G, int64_t gstride, int Hp, int Wp, const xv_params* p,
                           int64_t pu_gstride, const uint8_t* tu_log2, const int16_t* levels, const int16_t* mv,
                           int intra, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_params(p) || !valid_frame(G, Hp, Wp, p->ctu)) return XV_EINVAL;
    if (!recon || !tu_log2 || (!intra && (!levels || !mv))) {
        set_error("recon and tu_log2 (and levels and mv unless intra) are required");
        return XV_EINVAL;
    }
    if (!valid_planes(recon, recon, levels ? (const void*)levels : (const void*)recon, gstride)) return XV_EINVAL;
    DeviceGuard g(c->device);
    return deblock_into(c, recon, G, gstride, Hp, Wp, p, pu_gstride, tu_log2, levels, mv, intra, (cudaStream_t)stream);
}

xv_status xv_psnr(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* planes,
                  const uint16_t* recon, int Hp, int Wp, const double* minmax, double* psnr, double* mse,
                  uint64_t* sse10, double* mean, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (!planes || !recon || !minmax) { set_error("planes, recon and minmax are required"); return XV_EINVAL; }
    if (Hp < H || Wp < W) { set_error("plane %dx%d smaller than the cube %dx%d", Hp, Wp, H, W); return XV_EINVAL; }
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    xv_status s = ensure(c, c->bandq, sizeof(BandQ) * bands);
    if (s) return s;
    BandQ* bq = (BandQ*)c->bandq.ptr;
    c->launches += kLaunchBandq;
    if ((s = check_launch(xvh::launch_bandq(minmax, bands, bq, st), "band constants"))) return s;
    return psnr_into(c, src, dt, bands, T, H, W, planes, recon, Hp, Wp, bq, psnr, mse, sse10, mean, st);
}

xv_status xv_ssim(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* recon,
                  int Hp, int Wp, const double* minmax, double* ssim_band, double* ssim_mean, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (!recon || !minmax) { set_error("recon and minmax are required"); return XV_EINVAL; }
    if (Hp < H || Wp < W) { set_error("plane %dx%d smaller than the cube %dx%d", Hp, Wp, H, W); return XV_EINVAL; }
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = xvh::ssim_blocks_per_band(T, H, W);
    xv_status s;
    if ((s = ensure(c, c->bandq, sizeof(BandQ) * bands))) return s;
    if ((s = ensure(c, c->met_part, sizeof(xvh::MetricPart) * (size_t)nblk * bands))) return s;
    if ((s = ensure(c, c->met_out, sizeof(xvh::MetricPart) * bands))) return s;
    BandQ* bq = (BandQ*)c->bandq.ptr;
    c->launches += kLaunchBandq + 2;
    if ((s = check_launch(xvh::launch_bandq(minmax, bands, bq, st), "band constants"))) return s;
    if ((s = check_launch(xvh::launch_ssim(src, dt, bands, T, H, W, recon, Hp, Wp, bq, (xvh::MetricPart*)c->met_part.ptr,
                                           nblk, (xvh::MetricPart*)c->met_out.ptr, st),
                          "ssim")))
        return s;
    std::vector<xvh::MetricPart> out(bands);
    std::vector<BandQ> hq(bands);
    cudaError_t e = cudaMemcpyAsync(out.data(), c->met_out.ptr, sizeof(xvh::MetricPart) * bands, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hq.data(), bq, sizeof(BandQ) * bands, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "ssim read-back");
    double acc = 0.0;
    for (int b = 0; b < bands; ++b) {
        double v;
        if (hq[b].hi - hq[b].lo <= 0.0) v = (H >= 11 && W >= 11) ? 1.0 : NAN;  // a constant band
        else v = out[b].n > 0 ? out[b].sum / (double)out[b].n : NAN;
        if (ssim_band) ssim_band[b] = v;
        acc += v;
    }
    if (ssim_mean) *ssim_mean = acc / bands;
    return XV_OK;
}

xv_status xv_sa(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, const uint16_t* recon,
                int Hp, int Wp, const double* minmax, double* sa, int64_t* npix, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (!recon || !minmax) { set_error("recon and minmax are required"); return XV_EINVAL; }
    if (Hp < H || Wp < W) { set_error("plane %dx%d smaller than the cube %dx%d", Hp, Wp, H, W); return XV_EINVAL; }
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = xvh::sa_blocks((int64_t)T * H * W);
    xv_status s;
    if ((s = ensure(c, c->bandq, sizeof(BandQ) * bands))) return s;
    if ((s = ensure(c, c->met_part, sizeof(xvh::MetricPart) * (size_t)nblk))) return s;
    if ((s = ensure(c, c->met_out, sizeof(xvh::MetricPart) * bands))) return s;
    BandQ* bq = (BandQ*)c->bandq.ptr;
    c->launches += kLaunchBandq + 2;
    if ((s = check_launch(xvh::launch_bandq(minmax, bands, bq, st), "band constants"))) return s;
    if ((s = check_launch(xvh::launch_sa(src, dt, bands, T, H, W, recon, Hp, Wp, bq, (xvh::MetricPart*)c->met_part.ptr,
                                         nblk, (xvh::MetricPart*)c->met_out.ptr, st),
                          "spectral angle")))
        return s;
    xvh::MetricPart out;
    cudaError_t e = cudaMemcpyAsync(&out, c->met_out.ptr, sizeof out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "spectral angle read-back");
    if (sa) *sa = out.n > 0 ? out.sum / (double)out.n : NAN;
    if (npix) *npix = (int64_t)out.n;
    return XV_OK;
}

xv_status xv_pca_fit(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, double* mean,
                     double* components, double* variance, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (!mean || !components || !variance) { set_error("mean, components and variance are required"); return XV_EINVAL; }
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t npix = (int64_t)T * H * W;
    const int nblk = xvh::pca_fit_blocks(npix);
    xv_status s;
    if ((s = ensure(c, c->pca_part, sizeof(double) * 136 * (size_t)nblk))) return s;
    double* part = (double*)c->pca_part.ptr;
    std::vector<double> h((size_t)136 * nblk);
    c->launches += 1;
    if ((s = check_launch(xvh::launch_pca_sums(src, dt, bands, npix, part, nblk, st), "pca sums"))) return s;
    cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * (XV_MAX_BANDS + 1) * nblk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "pca sums read-back");
    double cnt = 0.0, m[XV_MAX_BANDS] = {0};
    for (int k = 0; k < nblk; ++k) {  // in block order
        for (int b = 0; b < bands; ++b) m[b] += h[(size_t)k * (XV_MAX_BANDS + 1) + b];
        cnt += h[(size_t)k * (XV_MAX_BANDS + 1) + XV_MAX_BANDS];
    }
    if (cnt < 1.0) { set_error("no pixel has all bands finite"); return XV_EINVAL; }
    for (int b = 0; b < bands; ++b) m[b] /= cnt;
    c->launches += 1;
    if ((s = check_launch(xvh::launch_pca_cov(src, dt, bands, npix, m, part, nblk, st), "pca covariance"))) return s;
    e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 136 * nblk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "pca covariance read-back");
    std::vector<double> cov((size_t)bands * bands, 0.0);
    const int npair = bands * (bands + 1) / 2;
    for (int k = 0; k < nblk; ++k) {
        int pi = 0, pj = 0;
        for (int q = 0; q < npair; ++q) {
            const double v = h[(size_t)k * 136 + q];
            cov[(size_t)pi * bands + pj] += v;
            if (++pj == bands) { ++pi; pj = pi; }
        }
    }
    for (int i = 0; i < bands; ++i)
        for (int j = i; j < bands; ++j) {
            cov[(size_t)i * bands + j] /= cnt;
            cov[(size_t)j * bands + i] = cov[(size_t)i * bands + j];
        }
    for (int b = 0; b < bands; ++b) mean[b] = m[b];
    xvh::pca_eigen(bands, cov.data(), variance, components);
    return XV_OK;
}

xv_status xv_pca_project(xv_ctx* c, const void* src, xv_dtype dt, int bands, int T, int H, int W, const double* mean,
                         const double* components, int npc, float* dst, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_cube(src, dt, bands, T, H, W)) return XV_EINVAL;
    if (!mean || !components || !dst || npc < 1 || npc > bands) {
        set_error("mean, components, dst and 1 <= npc (%d) <= bands (%d) are required", npc, bands);
        return XV_EINVAL;
    }
    DeviceGuard g(c->device);
    c->launches += 1;
    return check_launch(xvh::launch_pca_project(src, dt, bands, npc, (int64_t)T * H * W, mean, components, dst,
                                                (cudaStream_t)stream),
                        "pca project");
}

xv_status xv_pca_inverse(xv_ctx* c, const float* z, int npc, int bands, int T, int H, int W, const double* mean,
                         const double* components, float* dst, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!z || !mean || !components || !dst || bands < 1 || bands > XV_MAX_BANDS || npc < 1 || npc > bands || T < 1 ||
        H < 1 || W < 1) {
        set_error("pca inverse: z, mean, components, dst, 1 <= npc (%d) <= bands (%d) <= %d and a cube are required",
                  npc, bands, XV_MAX_BANDS);
        return XV_EINVAL;
    }
    DeviceGuard g(c->device);
    c->launches += 1;
    return check_launch(xvh::launch_pca_inverse(z, npc, bands, (int64_t)T * H * W, mean, components, dst,
                                                (cudaStream_t)stream),
                        "pca inverse");
}

size_t xv_job_scratch_bytes(const xv_job* j) {
    if (!j) return 0;
    const int G = (j->bands + 2) / 3, ctu = j->p.ctu > 0 ? j->p.ctu : 8;
    const int64_t npu = (int64_t)(plane_dim(j->H, ctu) / ctu) * (plane_dim(j->W, ctu) / ctu);
    return (size_t)G * j->T * (npu * 4 + npu * 4 + 8) + 4096;
}

xv_status xv_split_groups(const xv_job* whole, const int* qp, xv_job* out, int* njobs) {
    if (!valid_job(whole)) return XV_EINVAL;
    if (!qp || !out || !njobs) { set_error("qp, out and njobs are required"); return XV_EINVAL; }
    const xv_job& j = *whole;
    const int G = (j.bands + 2) / 3, Hp = plane_dim(j.H, j.p.ctu), Wp = plane_dim(j.W, j.p.ctu);
    const int64_t npu = (int64_t)(Hp / j.p.ctu) * (Wp / j.p.ctu);
    const int64_t fsz = 3LL * Hp * Wp, band = (int64_t)j.T * j.H * j.W;
    const size_t esz = j.dtype == XV_F32 ? 4 : 2;
    for (int g = 0; g < G; ++g) {
        xv_job o = j;
        xv_status s = xv_params_init(&o.p, j.p.ctu, j.p.search_range, j.p.tu_mask, qp[g]);
        if (s) return s;
        o.p.flags = j.p.flags;
        o.bands = std::min(3, j.bands - 3 * g);
        o.src = (const char*)j.src + (size_t)(3 * g) * band * esz;
        if (j.minmax) o.minmax = j.minmax + 2 * 3 * g;
        o.planes = j.planes + (size_t)g * j.T * fsz;
        o.recon = j.recon + (size_t)g * j.T * fsz;
        if (j.mv) o.mv = j.mv + (size_t)g * j.T * npu * 2;
        if (j.cost) o.cost = j.cost + (size_t)g * j.T * npu;
        if (j.levels) o.levels = j.levels + (size_t)g * j.T * fsz;
        if (j.tu_log2) o.tu_log2 = j.tu_log2 + (size_t)g * j.T * npu;
        if (j.bits) o.bits = j.bits + (size_t)g * j.T;
        out[g] = o;
    }
    *njobs = G;
    return XV_OK;
}

xv_status xv_encode_cube(xv_ctx* c, const xv_job* j, xv_result* r, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_job(j)) return XV_EINVAL;
    if (!r) { set_error("result is NULL"); return XV_EINVAL; }
    if ((j->p.flags & XV_DEBLOCK) && (!j->levels || !j->tu_log2)) {
        set_error("deblocking (XV_DEBLOCK) needs the job's levels and tu_log2 buffers");
        return XV_EINVAL;
    }
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const xv_params& p = j->p;
    const int G = (j->bands + 2) / 3, Hp = plane_dim(j->H, p.ctu), Wp = plane_dim(j->W, p.ctu), T = j->T;
    const int64_t npu = (int64_t)(Hp / p.ctu) * (Wp / p.ctu);
    const int64_t fsz = 3LL * Hp * Wp;
    std::memset(r, 0, sizeof *r);
    xv_status s;
    double* minmax = j->minmax;
    if (!minmax) {
        if ((s = ensure(c, c->tmp_minmax, sizeof(double) * 2 * j->bands))) return s;
        minmax = (double*)c->tmp_minmax.ptr;
    }
    if ((s = ensure(c, c->bandq, sizeof(BandQ) * j->bands))) return s;
    BandQ* bq = (BandQ*)c->bandq.ptr;
    if ((s = prepare_bands(c, j->src, j->dtype, j->bands, T, j->H, j->W, minmax, j->minmax_fixed, bq, st))) return s;
    c->launches += kLaunchQuant;
    if ((s = check_launch(xvh::launch_quantize_pack(j->src, j->dtype, j->bands, T, j->H, j->W, Hp, Wp, bq, j->planes, st),
                          "quantize_pack")))
        return s;
    int16_t* mv = j->mv;
    if (!mv) {
        if ((s = ensure(c, c->tmp_mv, sizeof(int16_t) * 2 * npu * G * T))) return s;
        mv = (int16_t*)c->tmp_mv.ptr;
    }
    uint64_t* bits = j->bits;
    if (!bits) {
        if ((s = ensure(c, c->tmp_bits, sizeof(uint64_t) * G * T))) return s;
        bits = (uint64_t*)c->tmp_bits.ptr;
    }
    if ((s = ensure_err_word(c))) return s;
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(uint64_t) * G * T, st);
    for (int gi = 0; gi < G && e == cudaSuccess; ++gi) {  // frame 0 has no motion
        e = cudaMemsetAsync(mv + (int64_t)gi * T * npu * 2, 0, sizeof(int16_t) * 2 * npu, st);
        if (e == cudaSuccess && j->cost) e = cudaMemsetAsync(j->cost + (int64_t)gi * T * npu, 0, sizeof(uint32_t) * npu, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    for (int t = 0; t < T; ++t) {
        const uint16_t* cur = j->planes + t * fsz;
        const uint16_t* ref = t > 0 ? j->recon + (t - 1) * fsz : nullptr;
        const bool intra = !ref && (p.flags & XV_INTRA);
        if (intra) {  // frame 0 with intra prediction; its modes take the vectors' place
            uint64_t launched = 0;
            s = check_launch(xvh::launch_intra_frame(cur, G, T * fsz, Hp, Wp, &p, mv, T * npu, j->recon,
                                                     j->levels, j->tu_log2, bits, T, st, &launched),
                             "intra frame");
            c->launches += launched;
            if (s) return s;
        }
        if (!intra) c->launches += kLaunchTqr + (ref ? kLaunchMe : 0);
        if (ref) {
            const xvh::WindowMap wm = window_map(c, ref, Wp, Hp, T * fsz, G, p);
            if ((s = check_launch(xvh::launch_me_frame(cur, ref, G, T * fsz, Hp, Wp, &p, mv + t * npu * 2,
                                                       j->cost ? j->cost + t * npu : nullptr, nullptr, nullptr, T * npu, st,
                                                       nullptr, &wm, (int*)c->dev_err.ptr),
                                  "motion_search")))
                return s;
        }
        if (!intra &&
            (s = check_launch(xvh::launch_tqr_frame(cur, ref, mv + t * npu * 2, G, T * fsz, Hp, Wp, &p, T * npu,
                                                    j->recon + t * fsz, j->levels ? j->levels + t * fsz : nullptr,
                                                    j->tu_log2 ? j->tu_log2 + t * npu : nullptr, bits + t, T, st),
                              "transform_quant_recon")))
            return s;
        if ((p.flags & XV_DEBLOCK) &&
            (s = deblock_into(c, j->recon + t * fsz, G, T * fsz, Hp, Wp, &p, T * npu, j->tu_log2 + t * npu,
                              j->levels + t * fsz, mv + t * npu * 2, intra ? 1 : 0, st)))
            return s;
    }
    r->status = XV_OK;
    if ((s = psnr_into(c, j->src, j->dtype, j->bands, T, j->H, j->W, j->planes, j->recon, Hp, Wp, bq, r->psnr_band,
                       r->mse_band, r->sse10_band, &r->psnr_mean, st)))
        return s;
    if ((s = fill_result(j, bits, G, r, st))) return s;
    if ((s = take_err_word(c))) r->status = s;
    return s;
}

}  // extern "C"

namespace {

// The batched paths' work stream and events (created on first use).
xv_status ensure_work_stream(xv_ctx* c) {
    if (c->work) return XV_OK;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) == cudaSuccess &&
        (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)) == cudaSuccess &&
        (e = cudaEventCreate(&c->ev0)) == cudaSuccess)
        e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) return cuda_fail(e, "work stream");
    return XV_OK;
}

xv_status ensure_side_streams(xv_ctx* c) {
    cudaError_t e = cudaSuccess;
    if (!c->fork_ev) e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) {
        if (!c->side[k]) e = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !c->side_ev[k]) e = cudaEventCreateWithFlags(&c->side_ev[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "side streams");
    return XV_OK;
}

xv_status ensure_upload_stream(xv_ctx* c, int njobs) {
    cudaError_t e = cudaSuccess;
    if (!c->up_st) e = cudaStreamCreateWithFlags(&c->up_st, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->up_join) e = cudaEventCreateWithFlags(&c->up_join, cudaEventDisableTiming);
    while (e == cudaSuccess && (int)c->up_ev.size() < njobs) {
        cudaEvent_t ev = nullptr;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) == cudaSuccess) c->up_ev.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(e, "upload stream");
    return XV_OK;
}

bool valid_djob(const xv_djob* j) {
    if (!j) { set_error("job is NULL"); return false; }
    if (!valid_params(&j->p) || !valid_frame(j->G, j->Hp, j->Wp, j->p.ctu)) return false;
    if (j->T < 1 || j->T > 65535) { set_error("T %d: must be in 1..65535", j->T); return false; }
    if (!j->levels || !j->mv || !j->tu_log2 || !j->recon) {
        set_error("levels, mv, tu_log2 and recon are required");
        return false;
    }
    if (!valid_planes(j->levels, j->recon, j->levels, 8)) return false;
    if (j->dst) {
        if (j->bands < 1 || j->bands > 3 * j->G || j->bands > XV_MAX_BANDS || j->H < 1 || j->W < 1 || j->H > j->Hp ||
            j->W > j->Wp || !j->minmax) {
            set_error("unpack: bands %d (1..min(3G, %d)), cube %dx%d inside %dx%d, and minmax are required", j->bands,
                      XV_MAX_BANDS, j->H, j->W, j->Hp, j->Wp);
            return false;
        }
    }
    return true;
}

}  // namespace

// xv_encode_batch, and with `host_src` (HOST [njobs], entries may be NULL)
// xv_encode_batch_from_host: job i's cube is first copied from host_src[i]
// to its src.  In the per-frame mode the copies of pinned cubes run on their
// own stream, smallest cube first, and each job's setup and chain wait only
// for its own cube, so the uploads overlap the encoding of the jobs already
// on the device; otherwise they precede the batch on its stream.
static xv_status encode_batch_impl(xv_ctx* c, const xv_job* jobs, int njobs, xv_result* results, void* stream,
                                   const void* const* host_src) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (njobs < 1 || njobs > 255 || !jobs || !results) { set_error("njobs %d: must be 1..255 with jobs and results", njobs); return XV_EINVAL; }
    for (int i = 0; i < njobs; ++i)
        if (!valid_job(&jobs[i]) || !no_options(&jobs[i].p, "xv_encode_batch")) return XV_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t caller = (cudaStream_t)stream;
    xv_status s;
    cudaError_t e = cudaSuccess;
    if ((s = ensure_work_stream(c))) return s;
    cudaStream_t st = c->work;

    // ---- geometry, descriptors, queue layout (host)
    const int ctus[4] = {8, 16, 32, 64};
    std::vector<xvh::JobDev> jd(njobs);
    std::vector<int64_t> bits_off(njobs), row_off(njobs), part_off(njobs), mv_off(njobs);
    std::vector<int> nblk(njobs);
    int64_t nbits = 0, nrows = 0, nparts = 0, nmv = 0;
    size_t total[4] = {0, 0, 0, 0}, nfirst[4] = {0, 0, 0, 0}, smem[4] = {0, 0, 0, 0};
    std::string shape[4];
    for (int i = 0; i < njobs; ++i) {
        const xv_job& j = jobs[i];
        const int G = (j.bands + 2) / 3, Hp = plane_dim(j.H, j.p.ctu), Wp = plane_dim(j.W, j.p.ctu);
        bits_off[i] = nbits;
        nbits += (int64_t)G * j.T;
        row_off[i] = nrows;
        nrows += (int64_t)G * j.T * (Hp / j.p.ctu);
        nblk[i] = xvh::psnr_blocks_per_band((int64_t)j.T * j.H * j.W, j.bands);
        part_off[i] = nparts;
        nparts += (int64_t)nblk[i] * j.bands;
        mv_off[i] = nmv;
        if (!j.mv) nmv += (int64_t)G * j.T * (Hp / j.p.ctu) * (Wp / j.p.ctu) * 2;
        const int k = j.p.ctu == 8 ? 0 : j.p.ctu == 16 ? 1 : j.p.ctu == 32 ? 2 : 3;
        const int64_t npu = (int64_t)(Hp / j.p.ctu) * (Wp / j.p.ctu);
        total[k] += (size_t)G * j.T * npu;
        nfirst[k] += (size_t)G * npu;
        smem[k] = std::max(smem[k], xvh::persist_smem_bytes(j.p.ctu, j.p.search_range, j.T > 1));
        char sh[96];
        snprintf(sh, sizeof sh, "%d:%d:%d:%d:%d:%d;", G, j.T, Hp, Wp, j.p.search_range, j.T > 1);
        shape[k] += sh;
    }
    size_t total_items = 0;
    xvh::ClassDev cls[4];
    for (int k = 0; k < 4; ++k) {
        cls[k] = xvh::ClassDev{(int64_t)total_items, (unsigned)total[k], (unsigned)nfirst[k]};
        total_items += total[k];
    }
    if (total_items > 0xffffffffu) { set_error("too many work items in one batch"); return XV_EINVAL; }
    if ((s = ensure(c, c->b_jobs, sizeof(xvh::JobDev) * njobs))) return s;
    if ((s = ensure(c, c->b_bits, sizeof(uint64_t) * nbits))) return s;
    if ((s = ensure(c, c->b_rowdone, sizeof(unsigned) * nrows))) return s;
    if ((s = ensure(c, c->b_depcnt, sizeof(unsigned) * nrows))) return s;
    if ((s = ensure(c, c->b_bandq, sizeof(BandQ) * XV_MAX_BANDS * njobs))) return s;
    if ((s = ensure(c, c->b_minmax, sizeof(double) * 2 * XV_MAX_BANDS * njobs))) return s;
    if ((s = ensure(c, c->b_ctl, sizeof(xvh::BatchCtl) * 4))) return s;
    if ((s = ensure(c, c->b_cls, sizeof(xvh::ClassDev) * 4))) return s;
    if ((s = ensure(c, c->b_items, sizeof(uint64_t) * total_items))) return s;
    if ((s = ensure(c, c->b_part, sizeof(xvh::PsnrPart) * nparts))) return s;
    if ((s = ensure(c, c->b_out, sizeof(xvh::PsnrPart) * XV_MAX_BANDS * njobs))) return s;
    if ((s = ensure(c, c->b_totals, sizeof(unsigned long long) * njobs))) return s;
    if ((s = ensure(c, c->b_mm_enc, sizeof(unsigned) * 2 * XV_MAX_BANDS * njobs))) return s;
    if ((s = ensure(c, c->b_mv, sizeof(int16_t) * (nmv > 0 ? nmv : 1)))) return s;
    if ((s = ensure(c, c->b_exact, sizeof(unsigned long long)))) return s;
    if ((s = ensure_side_streams(c))) return s;
    if ((s = ensure_err_word(c))) return s;
    // host uploads: bytes per job, and the order of the overlapped copies
    std::vector<size_t> up_bytes(njobs, 0);
    std::vector<int> up_order;
    if (host_src) {
        if ((s = ensure_upload_stream(c, njobs))) return s;
        for (int i = 0; i < njobs; ++i) {
            if (!host_src[i]) continue;
            const xv_job& j = jobs[i];
            up_bytes[i] = (size_t)j.bands * j.T * j.H * j.W * (j.dtype == XV_F32 ? 4 : 2);
            up_order.push_back(i);
        }
        std::stable_sort(up_order.begin(), up_order.end(), [&](int a, int b) { return up_bytes[a] < up_bytes[b]; });
    }
    auto upload = [&](int i, cudaStream_t us) -> xv_status {
        cudaError_t ue = cudaMemcpyAsync(const_cast<void*>(jobs[i].src), host_src[i], up_bytes[i],
                                         cudaMemcpyHostToDevice, us);
        return ue == cudaSuccess ? XV_OK : cuda_fail(ue, "host cube upload");
    };
    // copies from pageable memory cannot be captured: those batches copy
    // everything on the batch stream first, outside the graphs
    std::vector<int> pre_upload;
    for (int i : up_order) {
        cudaPointerAttributes pa{};
        const bool pinned = cudaPointerGetAttributes(&pa, host_src[i]) == cudaSuccess && pa.type == cudaMemoryTypeHost;
        if (!pinned) {
            (void)cudaGetLastError();
            pre_upload.swap(up_order);
            break;
        }
    }
    const size_t stage_bytes = sizeof(xvh::BatchCtl) * 4 + sizeof(unsigned long long) * njobs +
                               (sizeof(xvh::PsnrPart) + sizeof(BandQ)) * XV_MAX_BANDS * njobs + sizeof(unsigned long long);
    if (c->h_stage_bytes < stage_bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        if ((e = cudaMallocHost(&c->h_stage, stage_bytes)) != cudaSuccess) return cuda_fail(e, "pinned staging");
        c->h_stage_bytes = stage_bytes;
    }
    uint64_t* bits_all = (uint64_t*)c->b_bits.ptr;
    BandQ* bq_all = (BandQ*)c->b_bandq.ptr;
    double* mm_all = (double*)c->b_minmax.ptr;
    size_t qnext[4];
    for (int k = 0; k < 4; ++k) qnext[k] = (size_t)cls[k].qoff;
    for (int i = 0; i < njobs; ++i) {
        const xv_job& j = jobs[i];
        xvh::JobDev& d = jd[i];
        const int G = (j.bands + 2) / 3, Hp = plane_dim(j.H, j.p.ctu), Wp = plane_dim(j.W, j.p.ctu);
        const int k = j.p.ctu == 8 ? 0 : j.p.ctu == 16 ? 1 : j.p.ctu == 32 ? 2 : 3;
        d.planes = j.planes;
        d.recon = j.recon;
        d.mv = j.mv;
        d.cost = j.cost;
        d.levels = j.levels;
        d.tu = j.tu_log2;
        d.bits = j.bits ? j.bits : bits_all + bits_off[i];
        d.rowdone = (unsigned*)c->b_rowdone.ptr + row_off[i];
        d.depcnt = (unsigned*)c->b_depcnt.ptr + row_off[i];
        d.lf8 = j.p.lambda_fp8;
        d.lmv = j.p.lambda_mv_fp16;
        d.G = G; d.T = j.T; d.Hp = Hp; d.Wp = Wp; d.ctu = j.p.ctu; d.R = j.p.search_range; d.qp = j.p.qp;
        d.tu_mask = j.p.tu_mask;
        d.nx = Wp / j.p.ctu;
        d.ny = Hp / j.p.ctu;
        d.qfirst = (int64_t)qnext[k];
        d.tb = 0;
        d.te = j.T;
        qnext[k] += (size_t)G * d.nx * d.ny;
    }
    // descriptors go up before (and outside) the captured work
    e = cudaMemcpyAsync(c->b_jobs.ptr, jd.data(), sizeof(xvh::JobDev) * njobs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->b_cls.ptr, cls, sizeof cls, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptors");
    const xvh::JobDev* jobs_dev = (const xvh::JobDev*)c->b_jobs.ptr;
    unsigned char* hs = (unsigned char*)c->h_stage;
    xvh::BatchCtl* h_ctl = (xvh::BatchCtl*)hs;
    unsigned long long* h_tot = (unsigned long long*)(hs + sizeof(xvh::BatchCtl) * 4);
    xvh::PsnrPart* h_out = (xvh::PsnrPart*)(h_tot + njobs);
    BandQ* h_bq = (BandQ*)(h_out + XV_MAX_BANDS * njobs);
    unsigned long long* h_exact = (unsigned long long*)(h_bq + XV_MAX_BANDS * njobs);

    // ---- the batch as three stream-ordered, capturable parts: setup,
    // persistent kernels, results; the timing events go between them
    // job i's min/max, quantiser constants and planes, on stream ss (its own
    // min/max scratch, so that jobs can run this concurrently)
    auto job_setup = [&](int i, cudaStream_t ss) -> xv_status {
        const xv_job& j = jobs[i];
        double* mm = j.minmax ? j.minmax : mm_all + 2 * XV_MAX_BANDS * i;
        BandQ* bq = bq_all + XV_MAX_BANDS * i;
        xv_status r = prepare_bands(c, j.src, j.dtype, j.bands, j.T, j.H, j.W, mm, j.minmax_fixed, bq, ss,
                                    (unsigned*)c->b_mm_enc.ptr + 2 * XV_MAX_BANDS * i);
        if (r) return r;
        c->launches += kLaunchQuant;
        return check_launch(xvh::launch_quantize_pack(j.src, j.dtype, j.bands, j.T, j.H, j.W, jd[i].Hp, jd[i].Wp, bq,
                                                      j.planes, ss),
                            "quantize_pack");
    };
    // with_jobs: the host uploads and every job's setup here, on the batch
    // stream (else part_frames runs them per job, overlapped)
    auto part_setup = [&](bool with_jobs) -> xv_status {
        for (size_t k = 0; with_jobs && k < up_order.size(); ++k) {
            xv_status r = upload(up_order[k], st);
            if (r) return r;
        }
        for (int i = 0; with_jobs && i < njobs; ++i) {
            xv_status r = job_setup(i, st);
            if (r) return r;
        }
        c->launches += 1;
        xv_status r = check_launch(xvh::launch_batch_prologue(jobs_dev, njobs, (const xvh::ClassDev*)c->b_cls.ptr,
                                                              (uint64_t*)c->b_items.ptr, (xvh::BatchCtl*)c->b_ctl.ptr,
                                                              c->wait_budget, c->stall_row, st),
                                   "batch prologue");
        return r;
    };
    // the per-frame mode runs the whole batch when any CTU class with work is
    // tuned (or forced) to it
    auto frames_mode = [&](const int nt[4]) {
        for (int k = 0; k < 4; ++k)
            if (total[k] && nt[k] == kFramesMode) return true;
        return false;
    };
    auto run_frames = [&](bool overlap_up) -> xv_status {
        cudaError_t err = cudaSuccess;
        unsigned long long* exact = (unsigned long long*)c->b_exact.ptr;
        for (int i = 0; i < njobs; ++i) {
            const xv_job& j = jobs[i];
            cudaStream_t ss = c->side[i % kSideStreams];
            if (overlap_up) {  // every upload into the job's cube (its own, or another job's into the same buffer), then its setup
                const char* a0 = static_cast<const char*>(j.src);
                const char* a1 = a0 + (size_t)j.bands * j.T * j.H * j.W * (j.dtype == XV_F32 ? 4 : 2);
                for (int u : up_order) {
                    const char* b0 = static_cast<const char*>(jobs[u].src);
                    if (b0 < a1 && a0 < b0 + up_bytes[u] && (err = cudaStreamWaitEvent(ss, c->up_ev[u], 0)) != cudaSuccess)
                        return cuda_fail(err, "upload wait");
                }
                xv_status r = job_setup(i, ss);
                if (r) return r;
            }
            const int G = jd[i].G, T = j.T, Hp = jd[i].Hp, Wp = jd[i].Wp;
            const int64_t npu = (int64_t)jd[i].nx * jd[i].ny, fsz = 3LL * Hp * Wp;
            int16_t* mv = j.mv ? j.mv : (int16_t*)c->b_mv.ptr + mv_off[i];
            for (int g = 0; g < G && err == cudaSuccess; ++g) {  // frame 0 has no motion
                err = cudaMemsetAsync(mv + (int64_t)g * T * npu * 2, 0, sizeof(int16_t) * 2 * npu, ss);
                if (err == cudaSuccess && j.cost)
                    err = cudaMemsetAsync(j.cost + (int64_t)g * T * npu, 0, sizeof(uint32_t) * npu, ss);
            }
            if (err != cudaSuccess) return cuda_fail(err, "frame 0 vectors");
            for (int t = 0; t < T; ++t) {
                const uint16_t* cur = j.planes + t * fsz;
                const uint16_t* ref = t > 0 ? j.recon + (t - 1) * fsz : nullptr;
                xv_status r;
                if (ref) {
                    c->launches += kLaunchMe;
                    const xvh::WindowMap wm = window_map(c, ref, Wp, Hp, T * fsz, G, j.p);
                    if ((r = check_launch(xvh::launch_me_frame(cur, ref, G, T * fsz, Hp, Wp, &j.p, mv + t * npu * 2,
                                                               j.cost ? j.cost + t * npu : nullptr, nullptr, nullptr,
                                                               T * npu, ss, exact, &wm, (int*)c->dev_err.ptr),
                                          "motion_search")))
                        return r;
                }
                c->launches += kLaunchTqr;
                if ((r = check_launch(xvh::launch_tqr_frame(cur, ref, mv + t * npu * 2, G, T * fsz, Hp, Wp, &j.p, T * npu,
                                                            j.recon + t * fsz, j.levels ? j.levels + t * fsz : nullptr,
                                                            j.tu_log2 ? j.tu_log2 + t * npu : nullptr,
                                                            jd[i].bits + t, T, ss),
                                      "transform_quant_recon")))
                    return r;
            }
        }
        return XV_OK;
    };
    // the per-frame mode: job i's frames on side stream i mod 16 (motion
    // search, then transform per frame, as xv_encode_cube runs them), forked
    // from and joined back into the work stream by events (capturable).  The
    // side streams are joined even when a launch fails, so that no work of
    // the batch is left running after the call returns (and a capture stays
    // well formed).
    auto part_frames = [&](bool overlap_up) -> xv_status {
        cudaError_t err = cudaMemsetAsync(c->b_exact.ptr, 0, sizeof(unsigned long long), st);
        if (err == cudaSuccess) err = cudaEventRecord(c->fork_ev, st);
        const int nside = njobs < kSideStreams ? njobs : kSideStreams;
        int forked = 0;  // side streams that joined the fork
        for (int k = 0; k < nside && err == cudaSuccess; ++k)
            if ((err = cudaStreamWaitEvent(c->side[k], c->fork_ev, 0)) == cudaSuccess) forked = k + 1;
        // the host uploads, smallest cube first, each announcing its job's cube
        bool up_forked = false;
        xv_status r = XV_OK;
        if (err == cudaSuccess && overlap_up) {
            if ((err = cudaStreamWaitEvent(c->up_st, c->fork_ev, 0)) == cudaSuccess) up_forked = true;
            for (size_t k = 0; err == cudaSuccess && !r && k < up_order.size(); ++k) {
                if ((r = upload(up_order[k], c->up_st))) break;
                err = cudaEventRecord(c->up_ev[up_order[k]], c->up_st);
            }
        }
        if (!r) r = err != cudaSuccess ? cuda_fail(err, "fork") : run_frames(overlap_up);
        cudaError_t je = cudaSuccess;
        if (up_forked) {
            cudaError_t a = cudaEventRecord(c->up_join, c->up_st);
            if (a == cudaSuccess) a = cudaStreamWaitEvent(st, c->up_join, 0);
            je = a;
        }
        for (int k = 0; k < forked; ++k) {
            cudaError_t a = cudaEventRecord(c->side_ev[k], c->side[k]);
            if (a == cudaSuccess) a = cudaStreamWaitEvent(st, c->side_ev[k], 0);
            if (je == cudaSuccess) je = a;
        }
        if (r) return r;
        if (je != cudaSuccess) return cuda_fail(je, "join");
        c->batch_nt = kFramesMode;
        for (int k = 0; k < 4; ++k) c->batch_cfg[k] = total[k] ? kFramesMode : 0;
        return XV_OK;
    };
    // the persistent launch of CTU class k in configuration `code`
    auto launch_class = [&](int k, int code) -> xv_status {
        const int bnt = cfg_nt(code);
        const int grid = xvh::persist_grid(ctus[k], bnt, smem[k], false, cfg_per(code));
        xv_status r = check_launch(xvh::launch_persist(ctus[k], bnt, false, jobs_dev,
                                                       (uint64_t*)c->b_items.ptr + cls[k].qoff,
                                                       (xvh::BatchCtl*)c->b_ctl.ptr + k, smem[k], grid, st),
                                   "persistent encode");
        if (r) return r;
        c->launches += kLaunchPersist;
        c->batch_nt = bnt;
        c->batch_cfg[k] = code;
        return XV_OK;
    };
    // the per-frame mode of a batch with pinned host sources overlaps their uploads
    auto overlap_up = [&](const int nt[4]) { return !up_order.empty() && frames_mode(nt); };
    auto part_kernels = [&](const int nt[4]) -> xv_status {
        if (frames_mode(nt)) return part_frames(overlap_up(nt));
        xv_status r = XV_OK;
        for (int k = 0; k < 4; ++k) {
            if (!total[k]) continue;
            if ((r = launch_class(k, nt[k]))) return r;
        }
        return r;
    };
    auto part_results = [&]() -> xv_status {
        xv_status r = XV_OK;
        cudaError_t err = cudaSuccess;
        for (int i = 0; i < njobs; ++i) {
            const xv_job& j = jobs[i];
            c->launches += kLaunchPsnr;
            r = check_launch(xvh::launch_psnr(j.src, j.dtype, j.bands, j.T, j.H, j.W, j.planes, j.recon, jd[i].Hp,
                                              jd[i].Wp, bq_all + XV_MAX_BANDS * i,
                                              (xvh::PsnrPart*)c->b_part.ptr + part_off[i], nblk[i],
                                              (xvh::PsnrPart*)c->b_out.ptr + XV_MAX_BANDS * i, st),
                             "psnr");
            if (r) return r;
        }
        c->launches += 1;
        r = check_launch(xvh::launch_bits_totals(jobs_dev, njobs, (unsigned long long*)c->b_totals.ptr, st),
                         "bits totals");
        if (r) return r;
        err = cudaMemcpyAsync(h_ctl, c->b_ctl.ptr, sizeof(xvh::BatchCtl) * 4, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h_tot, c->b_totals.ptr, sizeof(unsigned long long) * njobs, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h_out, c->b_out.ptr, sizeof(xvh::PsnrPart) * XV_MAX_BANDS * njobs,
                                  cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h_bq, bq_all, sizeof(BandQ) * XV_MAX_BANDS * njobs, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h_exact, c->b_exact.ptr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (err != cudaSuccess) return cuda_fail(err, "batch results");
        return XV_OK;
    };
    auto body = [&](const int nt[4]) -> xv_status {
        xv_status r = part_setup(!overlap_up(nt));
        cudaError_t err;
        if (!r && (err = cudaEventRecord(c->ev0, st)) != cudaSuccess) r = cuda_fail(err, "event");
        if (!r) r = part_kernels(nt);
        if (!r && (err = cudaEventRecord(c->ev1, st)) != cudaSuccess) r = cuda_fail(err, "event");
        if (!r) r = part_results();
        return r;
    };

    // order after the caller's stream
    if ((e = cudaEventRecord(c->ev_in, caller)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c->ev_in, 0)) != cudaSuccess)
        return cuda_fail(e, "stream order");
    for (int i : pre_upload)
        if ((s = upload(i, st))) return s;

    // ---- configuration per CTU class: forced, cached, or tuned now
    int nt[4] = {256, 256, 256, 256};
    bool tune = false;
    for (int k = 0; k < 4; ++k) {
        if (!total[k]) continue;
        auto it = c->tuned_nt.find(shape[k]);
        if (it == c->tuned_nt.end()) tune = true;
        else nt[k] = it->second;
    }
    // a forced block size still runs as captured graphs (like a tuned one);
    // the stalled-row hook runs uncaptured
    const bool debug = c->stall_row >= 0;
    if (c->force_nt) {
        for (int k = 0; k < 4; ++k) nt[k] = c->force_nt;
        tune = false;
    }
    if (tune && !debug) {
        // The autotuner.  Candidates: per CTU class, every block size the
        // persistent kernel is built for, with as many resident blocks per
        // SM as fit and with one fewer; for the whole batch, the per-frame
        // mode.  Each is timed as the CUDA graph it would replay (the batch
        // prologue, which resets the counters, then the candidate's
        // launches): one warm-up replay, then the median of three.  A
        // class's persistent launches are independent of the other classes',
        // so each class keeps its fastest configuration; the per-frame mode
        // wins when it beats the sum of those.
        if ((s = part_setup(true))) return s;  // the cubes, planes and counters every candidate reads
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "autotune setup");
        const uint64_t launches_before = c->launches;
        auto time_graph = [&](const std::function<xv_status()>& record, float* med) -> xv_status {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t te = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (te != cudaSuccess) return cuda_fail(te, "autotune capture");
            xv_status r = check_launch(xvh::launch_batch_prologue(jobs_dev, njobs, (const xvh::ClassDev*)c->b_cls.ptr,
                                                                  (uint64_t*)c->b_items.ptr, (xvh::BatchCtl*)c->b_ctl.ptr,
                                                                  c->wait_budget, c->stall_row, st),
                                       "batch prologue");
            if (!r) r = record();
            te = cudaStreamEndCapture(st, &graph);
            if (r) { if (graph) cudaGraphDestroy(graph); return r; }
            if (te != cudaSuccess) return cuda_fail(te, "autotune capture");
            te = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (te != cudaSuccess) return cuda_fail(te, "autotune instantiate");
            float ms[4] = {0.f, 0.f, 0.f, 0.f};
            for (int rep = 0; rep < 4 && te == cudaSuccess; ++rep) {
                if ((te = cudaEventRecord(c->ev0, st)) != cudaSuccess || (te = cudaGraphLaunch(exec, st)) != cudaSuccess ||
                    (te = cudaEventRecord(c->ev1, st)) != cudaSuccess || (te = cudaStreamSynchronize(st)) != cudaSuccess)
                    break;
                te = cudaEventElapsedTime(&ms[rep], c->ev0, c->ev1);
            }
            cudaGraphExecDestroy(exec);
            if (te != cudaSuccess) return cuda_fail(te, "autotune replay");
            std::sort(ms + 1, ms + 4);  // ms[0] is the warm-up
            *med = ms[2];
            return XV_OK;
        };
        float persist_total = 0.f;
        int best_code[4] = {0, 0, 0, 0};
        c->tune_log.clear();
        for (int k = 0; k < 4; ++k) {
            if (!total[k]) continue;
            float best = 1e30f;
            for (int bnt : xvh::kPersistBlockSizes) {
                const int maxper = xvh::persist_blocks_per_sm(ctus[k], bnt, smem[k], false);
                const int npers = maxper >= 2 ? 2 : 1;  // as many as fit, and one fewer
                for (int pi = 0; pi < npers; ++pi) {
                    const int per = pi == 0 ? 0 : maxper - 1;
                    const int code = cfg_code(bnt, per);
                    float ms = 0.f;
                    if ((s = time_graph([&]() { return launch_class(k, code); }, &ms))) return s;
                    char line[96];
                    snprintf(line, sizeof line, "ctu%d nt%d per%d %.3f;", ctus[k], bnt, per ? per : maxper, ms);
                    c->tune_log += line;
                    if (ms < best) { best = ms; best_code[k] = code; }
                }
            }
            persist_total += best;
        }
        float frames_ms = 0.f;
        if ((s = time_graph([&]() { return part_frames(false); }, &frames_ms))) return s;
        {
            char line[64];
            snprintf(line, sizeof line, "frames %.3f;", frames_ms);
            c->tune_log += line;
        }
        const bool frames = frames_ms < persist_total;
        for (int k = 0; k < 4; ++k) {
            if (!total[k]) continue;
            nt[k] = frames ? kFramesMode : best_code[k];
            c->tuned_nt[shape[k]] = nt[k];
            c->class_tuned[k] = best_code[k];  // the persistent kernel's best, also when the batch runs per frame
        }
        c->launches = launches_before;  // the candidates' launches are not the batch's
    }

    for (int k = 0; k < 4; ++k) c->batch_cfg[k] = total[k] ? (frames_mode(nt) ? kFramesMode : nt[k]) : 0;

    // ---- run: replay the captured graph of this exact batch, or capture it
    if (c->use_graph && !debug) {
        std::string key;
        char buf[256];
        for (int i = 0; i < njobs; ++i) {
            const xv_job& j = jobs[i];
            // every job field a captured launch reads, the lambdas and flags included
            // (the per-frame mode passes them to its launches as arguments)
            snprintf(buf, sizeof buf, "%p,%d,%d,%d,%d,%d,%d,%d,%u,%d,%lld,%lld,%u,%p,%d,%p,%p,%p,%p,%p,%p,%p;", j.src,
                     (int)j.dtype, j.bands, j.T, j.H, j.W, j.p.ctu, j.p.search_range, j.p.tu_mask, j.p.qp,
                     (long long)j.p.lambda_fp8, (long long)j.p.lambda_mv_fp16, (unsigned)j.p.flags, (void*)j.minmax,
                     j.minmax_fixed, (void*)j.planes, (void*)j.recon, (void*)j.mv, (void*)j.cost, (void*)j.levels,
                     (void*)j.tu_log2, (void*)j.bits);
            key += buf;
        }
        snprintf(buf, sizeof buf, "|%d,%d,%d,%d|%p,%p,%p,%p,%p,%p,%p,%p,%p,%p,%p,%p,%p,%p,%p|%lld", nt[0], nt[1], nt[2],
                 nt[3], c->b_jobs.ptr, c->b_bits.ptr, c->b_rowdone.ptr, c->b_depcnt.ptr, c->b_bandq.ptr, c->b_minmax.ptr,
                 c->b_ctl.ptr, c->b_cls.ptr, c->b_items.ptr, c->b_part.ptr, c->b_out.ptr, c->b_totals.ptr,
                 c->h_stage, c->b_mv.ptr, c->b_exact.ptr, c->wait_budget);
        key += "|" + std::to_string(c->tma_polls) + (c->tma_off ? "n" : "t");
        for (int i = 0; host_src && i < njobs; ++i) {  // the uploads' sources
            snprintf(buf, sizeof buf, "h%p;", host_src[i]);
            key += buf;
        }
        key += buf;
        if (!c->graph[0] || key != c->graph_key) {
            for (cudaGraphExec_t& gx : c->graph)
                if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
            const uint64_t launches_before = c->launches;
            for (int part = 0; part < 3; ++part) {
                cudaGraph_t graph = nullptr;
                if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                    return cuda_fail(e, "begin capture");
                xv_status r = part == 0 ? part_setup(!overlap_up(nt)) : part == 1 ? part_kernels(nt) : part_results();
                e = cudaStreamEndCapture(st, &graph);
                if (r) { if (graph) cudaGraphDestroy(graph); c->launches = launches_before; return r; }
                if (e != cudaSuccess) { c->launches = launches_before; return cuda_fail(e, "end capture"); }
                e = cudaGraphInstantiate(&c->graph[part], graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) { c->graph[part] = nullptr; c->launches = launches_before; return cuda_fail(e, "graph instantiate"); }
            }
            c->launches = launches_before;  // counted when the graphs run
            c->graph_key = key;
            c->graph_captures++;
        }
        if ((e = cudaGraphLaunch(c->graph[0], st)) != cudaSuccess || (e = cudaEventRecord(c->ev0, st)) != cudaSuccess ||
            (e = cudaGraphLaunch(c->graph[1], st)) != cudaSuccess || (e = cudaEventRecord(c->ev1, st)) != cudaSuccess ||
            (e = cudaGraphLaunch(c->graph[2], st)) != cudaSuccess)
            return cuda_fail(e, "graph launch");
        c->graph_launches++;
        c->launches += (uint64_t)njobs * (kLaunchMinmax + kLaunchQuant + kLaunchPsnr) + 2;
        if (frames_mode(nt)) {
            for (int i = 0; i < njobs; ++i) c->launches += (uint64_t)jobs[i].T * kLaunchTqr + (uint64_t)(jobs[i].T - 1) * kLaunchMe;
            c->batch_nt = kFramesMode;
        } else {
            for (int k = 0; k < 4; ++k) if (total[k]) { c->launches += kLaunchPersist; c->batch_nt = nt[k]; }
        }
        for (int i = 0; i < njobs; ++i)
            if (jobs[i].minmax_fixed) c->launches -= kLaunchMinmax - kLaunchBandq;
    } else {
        if ((s = body(nt))) return s;
    }
    if ((e = cudaEventRecord(c->ev_out, st)) != cudaSuccess || (e = cudaStreamWaitEvent(caller, c->ev_out, 0)) != cudaSuccess)
        return cuda_fail(e, "stream order");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "batch");
    float kms = 0.f;
    cudaError_t te = cudaEventElapsedTime(&kms, c->ev0, c->ev1);
    if (te == cudaSuccess) {
        c->batch_ms = kms;
    } else {
        c->batch_ms = -(double)te;  // timing unavailable; the error is not carried into later calls
        cudaGetLastError();
    }

    // ---- results (host)
    c->batch_exact = 0;
    c->batch_full = 0;
    if (frames_mode(nt)) {
        c->batch_exact = *h_exact;
    } else {
        for (int k = 0; k < 4; ++k)
            if (total[k]) c->batch_exact += h_ctl[k].exact_cand;
    }
    for (int i = 0; i < njobs; ++i) {
        const uint64_t side = 2 * (uint64_t)jobs[i].p.search_range + 1;
        c->batch_full += (uint64_t)jd[i].G * (uint64_t)(jobs[i].T - 1) * jd[i].nx * jd[i].ny * side * side;
    }
    if (frames_mode(nt) && (s = take_err_word(c))) {
        for (int i = 0; i < njobs; ++i) results[i].status = s;
        return s;
    }
    for (int k = 0; k < 4; ++k)
        if (!frames_mode(nt) && total[k] && h_ctl[k].err) {
            set_error("a dependency wait of the persistent encode (CTU %d) ran out of time", ctus[k]);
            for (int i = 0; i < njobs; ++i) results[i].status = XV_ETIMEOUT;
            return (xv_status)h_ctl[k].err;
        }
    for (int i = 0; i < njobs; ++i) {
        const xv_job& j = jobs[i];
        xv_result* r = &results[i];
        std::memset(r, 0, sizeof *r);
        double acc = 0.0;
        bool inf = false;
        for (int b = 0; b < j.bands; ++b) {
            const xvh::PsnrPart& o = h_out[XV_MAX_BANDS * i + b];
            const BandQ& q = h_bq[XV_MAX_BANDS * i + b];
            const double cnt = (double)o.count;
            const double m = cnt > 0 ? o.sse / cnt : 0.0;
            const double peak = q.hi > 0.0 ? q.hi : q.hi - q.lo;
            const double p = m > 0.0 ? 10.0 * std::log10(peak * peak / m) : INFINITY;
            r->psnr_band[b] = p;
            r->mse_band[b] = m;
            r->sse10_band[b] = o.sse10;
            if (std::isinf(p)) inf = true; else acc += p;
        }
        r->psnr_mean = inf ? INFINITY : acc / j.bands;
        r->total_bits = h_tot[i];
        r->bands = j.bands;
        r->bpppb = (double)h_tot[i] / ((double)j.H * j.W * j.T * j.bands);
        r->ctu = j.p.ctu;
        const int k = j.p.ctu == 8 ? 0 : j.p.ctu == 16 ? 1 : j.p.ctu == 32 ? 2 : 3;
        r->block_size = cfg_nt(c->batch_cfg[k]);
        r->status = XV_OK;
    }
    return XV_OK;
}

extern "C" {

xv_status xv_encode_batch(xv_ctx* c, const xv_job* jobs, int njobs, xv_result* results, void* stream) {
    return encode_batch_impl(c, jobs, njobs, results, stream, nullptr);
}

xv_status xv_encode_batch_from_host(xv_ctx* c, const xv_job* jobs, const void* const* host_src, int njobs,
                                    xv_result* results, void* stream) {
    return encode_batch_impl(c, jobs, njobs, results, stream, host_src);
}

xv_status xv_measure_peak(xv_ctx* c, int kind, double* rate, double* ms_out) {
    if (!c || !rate) { set_error("ctx and rate are required"); return XV_EINVAL; }
    if (kind < 0 || kind > 3) { set_error("kind %d: must be 0..3", kind); return XV_EINVAL; }
    DeviceGuard g(c->device);
    xv_status s;
    if ((s = ensure(c, c->peak_buf, sizeof(uint32_t) * (128 + 4096)))) return s;
    uint32_t host_in[128];
    for (int i = 0; i < 128; ++i) host_in[i] = 0x4B000000u | (uint32_t)((i * 733 + 91) & 1023);  // biased 10-bit samples
    uint32_t* in = (uint32_t*)c->peak_buf.ptr;
    cudaError_t e = cudaMemcpy(in, host_in, sizeof host_in, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "peak input");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "peak events");
    }
    const int iters = 100000;
    double best = 0.0, best_ms = 0.0;
    int threads = 0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
        if ((e = cudaEventRecord(e0, 0)) != cudaSuccess) break;
        if ((e = xvh::launch_peak(kind, in, iters, in + 128, &threads, 0)) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, 0)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        c->launches++;
        const double r = (double)threads * iters * xvh::peak_chains() / (ms * 1e-3);
        if (rep > 0 && r > best) { best = r; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "peak microbenchmark");
    *rate = best;
    if (ms_out) *ms_out = best_ms;
    return XV_OK;
}

xv_status xv_decode_frame(xv_ctx* c, const int16_t* levels, const uint16_t* ref, const int16_t* mv,
                          const uint8_t* tu_log2, int G, int64_t gstride, int Hp, int Wp, const xv_params* p,
                          int64_t pu_gstride, uint16_t* recon, uint64_t* bits, int64_t bits_gstride, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!valid_params(p) || !valid_frame(G, Hp, Wp, p->ctu)) return XV_EINVAL;
    const bool intra = !ref && (p->flags & XV_INTRA);
    if (!levels || !tu_log2 || !recon || !bits || ((ref || intra || (p->flags & XV_DEBLOCK)) && !mv)) {
        set_error("levels, tu_log2, recon, bits (and mv with ref or the options) are required");
        return XV_EINVAL;
    }
    if (!valid_planes(levels, ref ? ref : recon, recon, gstride)) return XV_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    xv_status s;
    if (intra) {  // frame 0 with intra prediction: the modes are in mv[cu][0]
        uint64_t launched = 0;
        s = check_launch(xvh::launch_intra_decode_frame(levels, G, gstride, Hp, Wp, p->ctu, p->qp, mv, pu_gstride,
                                                        tu_log2, recon, bits, bits_gstride, st, &launched),
                         "intra decode");
        c->launches += launched;
    } else {
        c->launches += 1;
        s = check_launch(xvh::launch_dec_frame(levels, ref, mv, tu_log2, G, gstride, Hp, Wp, p, pu_gstride, recon, bits,
                                               bits_gstride, st),
                         "decode_frame");
    }
    if (!s && (p->flags & XV_DEBLOCK))
        s = deblock_into(c, recon, G, gstride, Hp, Wp, p, pu_gstride, tu_log2, levels, mv, intra ? 1 : 0, st);
    return s;
}

xv_status xv_unpack(xv_ctx* c, const uint16_t* recon, int bands, int T, int H, int W, int Hp, int Wp,
                    const double* minmax, float* dst, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (!recon || !minmax || !dst) { set_error("recon, minmax and dst are required"); return XV_EINVAL; }
    if (bands < 1 || bands > XV_MAX_BANDS || T < 1 || H < 1 || W < 1 || Hp < H || Wp < W) {
        set_error("unpack: bands %d (1..%d), cube %dx%dx%d inside planes %dx%d", bands, XV_MAX_BANDS, T, H, W, Hp, Wp);
        return XV_EINVAL;
    }
    DeviceGuard g(c->device);
    c->launches += 1;
    return check_launch(xvh::launch_unpack(recon, bands, T, H, W, Hp, Wp, minmax, dst, (cudaStream_t)stream), "unpack");
}

xv_status xv_decode_batch(xv_ctx* c, const xv_djob* jobs, int njobs, uint64_t* total_bits, void* stream) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (njobs < 1 || njobs > 255 || !jobs) { set_error("njobs %d: must be 1..255 with jobs", njobs); return XV_EINVAL; }
    for (int i = 0; i < njobs; ++i)
        if (!valid_djob(&jobs[i]) || !no_options(&jobs[i].p, "xv_decode_batch")) return XV_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t caller = (cudaStream_t)stream;
    xv_status s;
    cudaError_t e = cudaSuccess;
    if ((s = ensure_work_stream(c))) return s;
    cudaStream_t st = c->work;

    // ---- descriptors and queue layout (host), as xv_encode_batch
    std::vector<xvh::JobDev> jd(njobs);
    std::vector<int64_t> bits_off(njobs), row_off(njobs);
    int64_t nbits = 0, nrows = 0;
    size_t total[4] = {0, 0, 0, 0}, nfirst[4] = {0, 0, 0, 0};
    const int ctus[4] = {8, 16, 32, 64};
    for (int i = 0; i < njobs; ++i) {
        const xv_djob& j = jobs[i];
        bits_off[i] = nbits;
        nbits += (int64_t)j.G * j.T;
        row_off[i] = nrows;
        nrows += (int64_t)j.G * j.T * (j.Hp / j.p.ctu);
        const int k = j.p.ctu == 8 ? 0 : j.p.ctu == 16 ? 1 : j.p.ctu == 32 ? 2 : 3;
        const int64_t npu = (int64_t)(j.Hp / j.p.ctu) * (j.Wp / j.p.ctu);
        total[k] += (size_t)j.G * j.T * npu;
        nfirst[k] += (size_t)j.G * npu;
    }
    size_t total_items = 0;
    xvh::ClassDev cls[4];
    for (int k = 0; k < 4; ++k) {
        cls[k] = xvh::ClassDev{(int64_t)total_items, (unsigned)total[k], (unsigned)nfirst[k]};
        total_items += total[k];
    }
    if (total_items > 0xffffffffu) { set_error("too many work items in one batch"); return XV_EINVAL; }
    if ((s = ensure(c, c->b_jobs, sizeof(xvh::JobDev) * njobs))) return s;
    if ((s = ensure(c, c->b_bits, sizeof(uint64_t) * nbits))) return s;
    if ((s = ensure(c, c->b_rowdone, sizeof(unsigned) * nrows))) return s;
    if ((s = ensure(c, c->b_depcnt, sizeof(unsigned) * nrows))) return s;
    if ((s = ensure(c, c->b_ctl, sizeof(xvh::BatchCtl) * 4))) return s;
    if ((s = ensure(c, c->b_cls, sizeof(xvh::ClassDev) * 4))) return s;
    if ((s = ensure(c, c->b_items, sizeof(uint64_t) * total_items))) return s;
    if ((s = ensure(c, c->b_totals, sizeof(unsigned long long) * njobs))) return s;
    const size_t stage_bytes = sizeof(xvh::BatchCtl) * 4 + sizeof(unsigned long long) * njobs;
    if (c->h_stage_bytes < stage_bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        if ((e = cudaMallocHost(&c->h_stage, stage_bytes)) != cudaSuccess) return cuda_fail(e, "pinned staging");
        c->h_stage_bytes = stage_bytes;
    }
    size_t qnext[4];
    for (int k = 0; k < 4; ++k) qnext[k] = (size_t)cls[k].qoff;
    for (int i = 0; i < njobs; ++i) {
        const xv_djob& j = jobs[i];
        xvh::JobDev& d = jd[i];
        const int k = j.p.ctu == 8 ? 0 : j.p.ctu == 16 ? 1 : j.p.ctu == 32 ? 2 : 3;
        d.planes = nullptr;
        d.recon = j.recon;
        d.mv = const_cast<int16_t*>(j.mv);
        d.cost = nullptr;
        d.levels = const_cast<int16_t*>(j.levels);
        d.tu = const_cast<uint8_t*>(j.tu_log2);
        d.bits = j.bits ? j.bits : (uint64_t*)c->b_bits.ptr + bits_off[i];
        d.rowdone = (unsigned*)c->b_rowdone.ptr + row_off[i];
        d.depcnt = (unsigned*)c->b_depcnt.ptr + row_off[i];
        d.lf8 = 0;
        d.lmv = 0;
        d.G = j.G; d.T = j.T; d.Hp = j.Hp; d.Wp = j.Wp; d.ctu = j.p.ctu; d.R = j.p.search_range; d.qp = j.p.qp;
        d.tu_mask = j.p.tu_mask;
        d.nx = j.Wp / j.p.ctu;
        d.ny = j.Hp / j.p.ctu;
        d.qfirst = (int64_t)qnext[k];
        d.tb = 0;
        d.te = j.T;
        qnext[k] += (size_t)j.G * d.nx * d.ny;
    }
    e = cudaMemcpyAsync(c->b_jobs.ptr, jd.data(), sizeof(xvh::JobDev) * njobs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->b_cls.ptr, cls, sizeof cls, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "decode descriptors");
    const xvh::JobDev* jobs_dev = (const xvh::JobDev*)c->b_jobs.ptr;
    xvh::BatchCtl* h_ctl = (xvh::BatchCtl*)c->h_stage;
    unsigned long long* h_tot = (unsigned long long*)((unsigned char*)c->h_stage + sizeof(xvh::BatchCtl) * 4);

    if ((e = cudaEventRecord(c->ev_in, caller)) != cudaSuccess || (e = cudaStreamWaitEvent(st, c->ev_in, 0)) != cudaSuccess)
        return cuda_fail(e, "stream order");
    c->launches += 1;
    if ((s = check_launch(xvh::launch_batch_prologue(jobs_dev, njobs, (const xvh::ClassDev*)c->b_cls.ptr,
                                                     (uint64_t*)c->b_items.ptr, (xvh::BatchCtl*)c->b_ctl.ptr,
                                                     c->wait_budget, c->stall_row, st),
                          "decode prologue")))
        return s;
    if ((e = cudaEventRecord(c->ev0, st)) != cudaSuccess) return cuda_fail(e, "event");
    for (int k = 0; k < 4; ++k) {
        if (!total[k]) continue;
        // measured: 128 threads for CTU 32 (its frames are wide), 512 for CTU 64, 256 otherwise
        const int nt = c->force_nt ? c->force_nt : (ctus[k] == 32 ? 128 : ctus[k] == 64 ? 512 : 256);
        const size_t smem = xvh::decode_smem_bytes(ctus[k]);
        const int grid = xvh::persist_grid(ctus[k], nt, smem, true);
        if ((s = check_launch(xvh::launch_persist(ctus[k], nt, true, jobs_dev, (uint64_t*)c->b_items.ptr + cls[k].qoff,
                                                  (xvh::BatchCtl*)c->b_ctl.ptr + k, smem, grid, st),
                              "persistent decode")))
            return s;
        c->launches += kLaunchPersist;
        c->batch_nt = nt;
    }
    if ((e = cudaEventRecord(c->ev1, st)) != cudaSuccess) return cuda_fail(e, "event");
    c->launches += 1;
    if ((s = check_launch(xvh::launch_bits_totals(jobs_dev, njobs, (unsigned long long*)c->b_totals.ptr, st),
                          "bits totals")))
        return s;
    for (int i = 0; i < njobs; ++i) {
        const xv_djob& j = jobs[i];
        if (!j.dst) continue;
        c->launches += 1;
        if ((s = check_launch(xvh::launch_unpack(j.recon, j.bands, j.T, j.H, j.W, j.Hp, j.Wp, j.minmax, j.dst, st),
                              "unpack")))
            return s;
    }
    e = cudaMemcpyAsync(h_ctl, c->b_ctl.ptr, sizeof(xvh::BatchCtl) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_tot, c->b_totals.ptr, sizeof(unsigned long long) * njobs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_out, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, c->ev_out, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "decode batch");
    float kms = 0.f;
    if (cudaEventElapsedTime(&kms, c->ev0, c->ev1) == cudaSuccess) c->batch_ms = kms;
    else { c->batch_ms = -1.0; cudaGetLastError(); }
    c->batch_exact = 0;
    c->batch_full = 0;
    for (int k = 0; k < 4; ++k)
        if (total[k] && h_ctl[k].err) {
            set_error("a dependency wait of the persistent decode (CTU %d) ran out of time", ctus[k]);
            return (xv_status)h_ctl[k].err;
        }
    if (total_bits)
        for (int i = 0; i < njobs; ++i) total_bits[i] = h_tot[i];
    return XV_OK;
}

xv_status xv_last_batch_block_size(const xv_ctx* c, int* nt) {
    if (!c || !nt) { set_error("ctx and nt are required"); return XV_EINVAL; }
    *nt = c->batch_nt;
    return XV_OK;
}

xv_status xv_last_batch_config(const xv_ctx* c, int ctu, int* block_size, int* blocks_per_sm) {
    if (!c || !block_size) { set_error("ctx and block_size are required"); return XV_EINVAL; }
    const int k = ctu == 8 ? 0 : ctu == 16 ? 1 : ctu == 32 ? 2 : ctu == 64 ? 3 : -1;
    if (k < 0) { set_error("ctu %d: must be 8, 16, 32 or 64", ctu); return XV_EINVAL; }
    *block_size = cfg_nt(c->batch_cfg[k]);
    if (blocks_per_sm) *blocks_per_sm = cfg_per(c->batch_cfg[k]);
    return XV_OK;
}

const char* xv_last_tune_log(const xv_ctx* c) { return c ? c->tune_log.c_str() : ""; }

xv_status xv_last_batch_search_stats(const xv_ctx* c, uint64_t* exact_candidates, uint64_t* full_candidates) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (exact_candidates) *exact_candidates = c->batch_exact;
    if (full_candidates) *full_candidates = c->batch_full;
    return XV_OK;
}

xv_status xv_last_batch_kernel_ms(const xv_ctx* c, double* ms) {
    if (!c || !ms) { set_error("ctx and ms are required"); return XV_EINVAL; }
    *ms = c->batch_ms;
    return XV_OK;
}

uint64_t xv_ctx_launches(const xv_ctx* c) { return c ? c->launches : 0; }

// Test hooks for the bounded device waits of the persistent path.
xv_status xv_debug_set_wait_budget(xv_ctx* c, long long cycles) {
    if (!c || cycles < 1) { set_error("bad wait budget"); return XV_EINVAL; }
    c->wait_budget = cycles;
    return XV_OK;
}

xv_status xv_serve_start(xv_ctx* c, int max_slots, int frames_per_tick) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (c->serve) { set_error("serving already started on this context"); return XV_EINVAL; }
    if (max_slots < 1 || max_slots > 255 || frames_per_tick < 1) {
        set_error("max_slots %d (1..255) / frames_per_tick %d (>= 1)", max_slots, frames_per_tick);
        return XV_EINVAL;
    }
    DeviceGuard g(c->device);
    xv_status st = XV_OK;
    // the persistent configuration per CTU class: the autotuner's latest
    // choice for that class on this context, else 256-thread blocks
    int block[4], per_cap[4];
    for (int k = 0; k < 4; ++k) {
        const int code = c->class_tuned[k];
        const bool persistent = code != 0 && code != kFramesMode;
        block[k] = persistent ? cfg_nt(code) : 256;
        per_cap[k] = persistent ? cfg_per(code) : 0;
    }
    xvh::ServeState* s = xvh::serve_create(c->device, max_slots, frames_per_tick, c->budget, c->wait_budget, block,
                                           per_cap, &st);
    if (st) { xvh::serve_destroy(s); return st; }
    c->serve = s;
    return XV_OK;
}

xv_status xv_serve_submit(xv_ctx* c, const xv_request* r, uint64_t* ticket) {
    if (!c || !c->serve) { set_error("serving not started"); return XV_EINVAL; }
    if (!r || !ticket) { set_error("request and ticket are required"); return XV_EINVAL; }
    if (!valid_cube(r->src, r->dtype, r->bands, r->T, r->H, r->W) || !valid_params(&r->p) ||
        !no_options(&r->p, "xv_serve_submit"))
        return XV_EINVAL;
    return xvh::serve_submit(c->serve, r, ticket);
}

xv_status xv_serve_poll(xv_ctx* c, uint64_t ticket, xv_result* res, int* done) {
    if (!c || !c->serve) { set_error("serving not started"); return XV_EINVAL; }
    if (!done) { set_error("done is required"); return XV_EINVAL; }
    return xvh::serve_poll(c->serve, ticket, res, done);
}

xv_status xv_serve_cancel(xv_ctx* c, uint64_t ticket) {
    if (!c || !c->serve) { set_error("serving not started"); return XV_EINVAL; }
    return xvh::serve_cancel(c->serve, ticket);
}

xv_status xv_serve_stats(xv_ctx* c, uint64_t* ticks, double* kernel_ms, int* peak, size_t* bytes) {
    if (!c || !c->serve) { set_error("serving not started"); return XV_EINVAL; }
    xvh::serve_stats(c->serve, ticks, kernel_ms, peak, bytes);
    return XV_OK;
}

xv_status xv_serve_stop(xv_ctx* c) {
    if (!c || !c->serve) { set_error("serving not started"); return XV_EINVAL; }
    DeviceGuard g(c->device);
    xvh::serve_destroy(c->serve);
    c->serve = nullptr;
    return XV_OK;
}

xv_status xv_batch_graph_stats(const xv_ctx* c, uint64_t* captures, uint64_t* launches) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    if (captures) *captures = c->graph_captures;
    if (launches) *launches = c->graph_launches;
    return XV_OK;
}

xv_status xv_set_batch_graphs(xv_ctx* c, int enable) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    c->use_graph = enable ? 1 : 0;
    return XV_OK;
}

xv_status xv_debug_force_block_size(xv_ctx* c, int nt) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    bool ok = nt == 0 || nt == kFramesMode;
    for (int v : xvh::kPersistBlockSizes) ok = ok || (nt >= 0 && cfg_nt(nt) == v && cfg_per(nt) <= 32);
    if (!ok) {
        set_error("block size %d is neither one the persistent kernel is built for nor %d (per-frame mode)", nt,
                  kFramesMode);
        return XV_EINVAL;
    }
    c->force_nt = nt;
    return XV_OK;
}

xv_status xv_debug_set_window_wait(xv_ctx* c, long long polls) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    c->tma_polls = polls > 0 ? polls : (1ll << 24);
    c->tma_off = polls < 0;
    return XV_OK;
}

xv_status xv_debug_stall_row(xv_ctx* c, long long row) {
    if (!c) { set_error("ctx is NULL"); return XV_EINVAL; }
    c->stall_row = row;
    return XV_OK;
}

}  // extern "C"
