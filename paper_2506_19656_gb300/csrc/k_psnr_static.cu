// k_psnr_static.cu -- xv_psnr_noalloc: the PSNR reduction with its scratch in a
// fixed device array instead of context allocations.
//
// For callers that cannot allocate device memory (see include/xv.h).  The
// per-block partial sums, the per-band quantiser constants and the per-band
// totals live in g_psnr_scratch, a file-scope device array of a fixed size
// that every GPU loading this library holds until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that
// device current) and every later call on the device reuses it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kMaxBlocksPerBand = 256;  // psnr_blocks_per_band never exceeds this
constexpr size_t kPartBytes = sizeof(PsnrPart) * (size_t)XV_MAX_BANDS * kMaxBlocksPerBand;
constexpr size_t kOutBytes = sizeof(PsnrPart) * XV_MAX_BANDS;
constexpr size_t kBandQBytes = sizeof(BandQ) * XV_MAX_BANDS;
constexpr size_t kScratchBytes = kPartBytes + kOutBytes + kBandQBytes;  // about 129 KB

static __device__ __align__(256) unsigned char g_psnr_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_psnr_scratch on the current device (set up once).
xv_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device %d: the fixed scratch supports devices 0..%d", dev, kMaxDevices - 1);
        return XV_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_psnr_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_psnr_scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return XV_OK;
}

}  // namespace
}  // namespace xvh

extern "C" xv_status xv_psnr_noalloc(const void* src, xv_dtype dt, int bands, int T, int H, int W,
                                     const uint16_t* planes, const uint16_t* recon, int Hp, int Wp,
                                     const double* minmax, double* psnr, double* mse, uint64_t* sse10,
                                     double* mean, void* stream) {
    using namespace xvh;
    if (!src || !planes || !recon || !minmax) {
        set_error("src, planes, recon and minmax are required");
        return XV_EINVAL;
    }
    if (dt != XV_F32 && dt != XV_U16) { set_error("dtype %d: must be XV_F32 or XV_U16", (int)dt); return XV_EINVAL; }
    if (bands < 1 || bands > XV_MAX_BANDS) {
        set_error("bands %d: the fixed scratch holds at most %d bands", bands, XV_MAX_BANDS);
        return XV_EINVAL;
    }
    if (T < 1 || H < 1 || W < 1 || Hp < H || Wp < W) {
        set_error("bad cube %dx%dx%d or planes %dx%d", T, H, W, Hp, Wp);
        return XV_EINVAL;
    }
    const int nblk = psnr_blocks_per_band((int64_t)T * H * W, bands);
    if (nblk > kMaxBlocksPerBand) {
        set_error("%d partial sums per band exceed the fixed scratch (%d)", nblk, kMaxBlocksPerBand);
        return XV_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* base = nullptr;
    xv_status s = scratch_address(dev, &base);
    if (s) return s;
    PsnrPart* part = reinterpret_cast<PsnrPart*>(base);
    PsnrPart* out = reinterpret_cast<PsnrPart*>(base + kPartBytes);
    BandQ* bq = reinterpret_cast<BandQ*>(base + kPartBytes + kOutBytes);
    cudaStream_t st = (cudaStream_t)stream;
    // every partial, total and constant is rewritten by this call: nothing
    // left by an earlier call is read
    if ((e = launch_bandq(minmax, bands, bq, st)) != cudaSuccess) return cuda_fail(e, "band constants");
    if ((e = launch_psnr(src, dt, bands, T, H, W, planes, recon, Hp, Wp, bq, part, nblk, out, st)) != cudaSuccess)
        return cuda_fail(e, "psnr");
    PsnrPart hout[XV_MAX_BANDS];
    BandQ hq[XV_MAX_BANDS];
    e = cudaMemcpyAsync(hout, out, sizeof(PsnrPart) * bands, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hq, bq, sizeof(BandQ) * bands, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "psnr read-back");
    double acc = 0.0;
    bool inf = false;
    for (int b = 0; b < bands; ++b) {
        const double cnt = (double)hout[b].count;
        const double m = cnt > 0 ? hout[b].sse / cnt : 0.0;
        const double peak = hq[b].hi > 0.0 ? hq[b].hi : hq[b].hi - hq[b].lo;
        const double p = m > 0.0 ? 10.0 * std::log10(peak * peak / m) : INFINITY;
        if (psnr) psnr[b] = p;
        if (mse) mse[b] = m;
        if (sse10) sse10[b] = hout[b].sse10;
        if (std::isinf(p)) inf = true; else acc += p;
    }
    if (mean) *mean = inf ? INFINITY : acc / bands;
    return XV_OK;
}
