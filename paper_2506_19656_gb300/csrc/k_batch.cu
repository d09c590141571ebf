// k_batch.cu -- the batched path: one persistent launch for every frame of
// every cube in a batch, scheduled by data flow.
//
// A work item is (job, group, frame, PU).  Items enter a device ready queue
// only when everything they read exists: the items of each job's first
// frame in the launch are queued by the prologue; a frame t+1 item is queued
// when the CTU rows of frame t that its
// motion search and compensation read (rows within R + 4 samples of the PU)
// are complete.  Each CTU row has a completion counter (PUs done); when a row
// completes, the block that finished it increments the dependency counters of
// the next frame's rows that read it, and the block that completes such a
// counter appends that row's items to the queue.  Blocks take queue positions
// in order with an atomic ticket, so a block only waits when no item is ready
// at all.  Every queued item depends only on finished items, so the queue
// always fills; each wait is still bounded by a cycle budget, after which the
// block records XV_ETIMEOUT and every block drains the queue without working.
//
// The reference planes are written during the launch, so they are read through
// L2 (no read-only cache); a finished item publishes its writes with a fence
// before its row counter is incremented, and queue slots are read with acquire
// loads.
#include <cuda_runtime.h>

#include <cstdint>

#include "batch.cuh"

namespace xvh {
batch::PersistFn persist_fn_ctu8(int nt, bool decode);
batch::PersistFn persist_fn_ctu16(int nt, bool decode);
batch::PersistFn persist_fn_ctu32(int nt, bool decode);
batch::PersistFn persist_fn_ctu64(int nt, bool decode);
namespace {

// Batch prologue: block j < njobs handles job j (its bits and counters over
// the window, the window's first-frame items); the others fill the empty
// queue slots; block njobs also writes the control blocks.
__global__ void k_batch_prologue(const JobDev* __restrict__ jobs, int njobs, const ClassDev* __restrict__ cls,
                                 uint64_t* queue, BatchCtl* ctl, long long budget, long long stall_row) {
    const int b = blockIdx.x;
    if (b < njobs) {
        const JobDev& J = jobs[b];
        const int64_t npu = (int64_t)J.nx * J.ny, nw = J.te - J.tb;
        for (int64_t i = threadIdx.x; i < (int64_t)J.G * nw; i += blockDim.x) {
            const int g = (int)(i / nw), t = J.tb + (int)(i - (int64_t)g * nw);
            J.bits[(int64_t)g * J.T + t] = 0ull;
        }
        for (int64_t i = threadIdx.x; i < (int64_t)J.G * nw * J.ny; i += blockDim.x) {
            const int64_t per_g = nw * J.ny;
            const int g = (int)(i / per_g);
            const int64_t o = ((int64_t)g * J.T + J.tb) * J.ny + (i - g * per_g);
            J.rowdone[o] = 0u;
            J.depcnt[o] = 0u;
        }
        for (int64_t i = threadIdx.x; i < (int64_t)J.G * npu; i += blockDim.x) {
            const int g = (int)(i / npu), pu = (int)(i - (int64_t)g * npu);
            queue[J.qfirst + i] = ((uint64_t)b << 56) | ((uint64_t)g << 48) | ((uint64_t)J.tb << 32) | (uint32_t)pu;
        }
        return;
    }
    const int64_t stride = (int64_t)(gridDim.x - njobs) * blockDim.x;
    const int64_t start = (int64_t)(b - njobs) * blockDim.x + threadIdx.x;
    for (int k = 0; k < 4; ++k) {
        const int64_t lo = cls[k].qoff + cls[k].nfirst, hi = cls[k].qoff + cls[k].total;
        for (int64_t i = lo + start; i < hi; i += stride) queue[i] = kEmptyItem;
    }
    if (b == njobs && threadIdx.x < 4) {
        const int k = threadIdx.x;
        ctl[k] = BatchCtl{0u, cls[k].nfirst, cls[k].total, 0, budget, stall_row, 0ull};
    }
}

__global__ void k_bits_totals(const JobDev* __restrict__ jobs, unsigned long long* totals) {
    const JobDev& J = jobs[blockIdx.x];
    const int64_t nb = (int64_t)J.G * J.T;
    unsigned long long s = 0;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) s += J.bits[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ unsigned long long red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        totals[blockIdx.x] = t;
    }
}

using batch::PersistFn;
PersistFn persist_fn(int ctu, int nt, bool decode) {
    switch (ctu) {
        case 8: return persist_fn_ctu8(nt, decode);
        case 16: return persist_fn_ctu16(nt, decode);
        case 32: return persist_fn_ctu32(nt, decode);
        case 64: return persist_fn_ctu64(nt, decode);
    }
    return nullptr;
}

}  // namespace

cudaError_t launch_batch_prologue(const JobDev* jobs, int njobs, const ClassDev* cls, uint64_t* queue,
                                  BatchCtl* ctl, long long budget, long long stall_row, cudaStream_t st) {
    k_batch_prologue<<<njobs + 64, 256, 0, st>>>(jobs, njobs, cls, queue, ctl, budget, stall_row);
    return cudaGetLastError();
}

cudaError_t launch_bits_totals(const JobDev* jobs, int njobs, unsigned long long* totals, cudaStream_t st) {
    k_bits_totals<<<njobs, 256, 0, st>>>(jobs, totals);
    return cudaGetLastError();
}

size_t decode_smem_bytes(int ctu) {
    size_t a = xvd::dec_smem_bytes(ctu), b = xvd::tqr_smem_bytes(ctu);
    return a > b ? a : b;
}

size_t persist_smem_bytes(int ctu, int R, bool has_me) {
    size_t a = xvd::tqr_smem_bytes(ctu);
    size_t b = has_me ? xvd::me_smem_bytes(ctu, R) : 0;
    return a > b ? a : b;
}

int persist_grid(int ctu, int nt, size_t smem, bool decode, int per_cap) {
    PersistFn fn = persist_fn(ctu, nt, decode);
    if (!fn) return 0;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nt, smem) != cudaSuccess) {
        cudaGetLastError();  // reported by the launch that follows, not left behind
        per = 1;
    }
    if (per_cap > 0 && per > per_cap) per = per_cap;
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_persist(int ctu, int nt, bool decode, const JobDev* jobs, uint64_t* queue, BatchCtl* ctl,
                           size_t smem, int grid, cudaStream_t st) {
    PersistFn fn = persist_fn(ctu, nt, decode);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, nt, smem, st>>>(jobs, queue, ctl);
    return cudaGetLastError();
}

}  // namespace xvh
