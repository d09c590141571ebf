// k_batch.cu -- the batched path: one persistent launch for every frame of
// every cube in a batch.
//
// Items (job, group, frame, PU) are taken from a device work queue in
// frame-major order by an atomic ticket.  An item of frame t first waits for
// the CTU rows of frame t-1 that its motion search and compensation read
// (rows within R + 4 samples of the PU); every dependency has a smaller
// ticket and was taken by a block that is running, so the waits always end.
// Each wait is still bounded by a cycle budget: when it runs out the block
// records XV_ETIMEOUT in the control block, and from then on every block
// skips its items, so the launch drains quickly and the host reports the
// error.  The reference is read through L2 (it is written during the
// launch); a finished item publishes its rows with a fence before its
// counter increment.
#include <cuda_runtime.h>

#include <cstdint>

#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

constexpr int kNT = 256;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

// Thread 0: wait until rows [r0, r1] of the previous frame are complete.
__device__ bool wait_rows(const unsigned* rowdone, int r0, int r1, unsigned need, BatchCtl* ctl) {
    const long long start = clock64();
    for (int r = r0; r <= r1; ++r) {
        while (ld_acquire(rowdone + r) < need) {
            if (ld_volatile_int(&ctl->err)) return false;
            if (clock64() - start > ctl->budget) {
                atomicCAS(&ctl->err, 0, (int)XV_ETIMEOUT);
                return false;
            }
            __nanosleep(100);
        }
    }
    return true;
}

template <int N>
__device__ void item_work(const JobDev& J, int g, int t, int pu, unsigned char* smem) {
    const int64_t plane = (int64_t)J.Hp * J.Wp, fsz = 3 * plane;
    const int64_t f = (int64_t)g * J.T + t;
    const uint16_t* cur = J.planes + f * fsz;
    const uint16_t* ref = t > 0 ? J.recon + (f - 1) * fsz : nullptr;
    const int x0 = (pu % J.nx) * N, y0 = (pu / J.nx) * N;
    xvd::MeResult m{0, 0, 0u, 0, 0, 0u};
    if (ref) m = xvd::me_pu<N, kNT, true>(cur, ref, J.Hp, J.Wp, x0, y0, J.R, J.lmv, smem);
    const int64_t npu = (int64_t)J.nx * J.ny;
    uint32_t b = xvd::tqr_cu<N, kNT, true>(cur, ref, plane, J.Hp, J.Wp, x0, y0, m.mvx, m.mvy, J.qp, J.tu_mask,
                                           J.lf8, J.recon + f * fsz, J.levels ? J.levels + f * fsz : nullptr,
                                           J.tu ? J.tu + f * npu + pu : nullptr, smem);
    if (threadIdx.x == 0) {
        const int64_t o = f * npu + pu;
        if (J.mv) { J.mv[2 * o] = (int16_t)m.mvx; J.mv[2 * o + 1] = (int16_t)m.mvy; }
        if (J.cost) J.cost[o] = m.cost;
        atomicAdd(reinterpret_cast<unsigned long long*>(J.bits + f), (unsigned long long)b);
    }
}

template <int N>
__global__ void __launch_bounds__(kNT)
k_persist(const JobDev* __restrict__ jobs, const uint64_t* __restrict__ items, unsigned nitems, BatchCtl* ctl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_item;
    __shared__ int s_go;
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned it = atomicAdd(&ctl->next, 1u);
            int go = 0;
            if (it < nitems && !ld_volatile_int(&ctl->err)) {
                const uint64_t key = items[it];
                const JobDev& J = jobs[key >> 56];
                const int g = (int)((key >> 48) & 0xff), t = (int)((key >> 32) & 0xffff), pu = (int)(uint32_t)key;
                go = 1;
                if (t > 0) {
                    const int y0 = (pu / J.nx) * N;
                    int r0 = (y0 - J.R - 4) / N, r1 = (y0 + N - 1 + J.R + 4) / N;
                    if (y0 - J.R - 4 < 0) r0 = 0;
                    if (r1 > J.ny - 1) r1 = J.ny - 1;
                    const unsigned need = (unsigned)J.nx + (it == ctl->stall_item ? 1u : 0u);
                    go = wait_rows(J.rowdone + ((int64_t)g * J.T + t - 1) * J.ny, r0, r1, need, ctl) ? 1 : 0;
                }
            }
            s_item = it;
            s_go = go;
        }
        __syncthreads();
        const unsigned it = s_item;
        if (it >= nitems) break;
        if (s_go) {
            const uint64_t key = items[it];
            const JobDev& J = jobs[key >> 56];
            const int g = (int)((key >> 48) & 0xff), t = (int)((key >> 32) & 0xffff), pu = (int)(uint32_t)key;
            item_work<N>(J, g, t, pu, smem);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0)
                atomicAdd(J.rowdone + ((int64_t)g * J.T + t) * J.ny + pu / J.nx, 1u);
        }
        __syncthreads();
    }
}

using PersistFn = void (*)(const JobDev*, const uint64_t*, unsigned, BatchCtl*);
PersistFn persist_fn(int ctu) {
    switch (ctu) {
        case 8: return k_persist<8>;
        case 16: return k_persist<16>;
        case 32: return k_persist<32>;
        case 64: return k_persist<64>;
    }
    return nullptr;
}

}  // namespace

size_t persist_smem_bytes(int ctu, int R, bool has_me) {
    size_t a = xvd::tqr_smem_bytes(ctu);
    size_t b = has_me ? xvd::me_smem_bytes(ctu, R) : 0;
    return a > b ? a : b;
}

int persist_grid(int ctu, size_t smem) {
    PersistFn fn = persist_fn(ctu);
    if (!fn) return 0;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kNT, smem);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_persist(int ctu, const JobDev* jobs, const uint64_t* items, unsigned nitems, BatchCtl* ctl,
                           size_t smem, int grid, cudaStream_t st) {
    PersistFn fn = persist_fn(ctu);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, kNT, smem, st>>>(jobs, items, nitems, ctl);
    return cudaGetLastError();
}

}  // namespace xvh
