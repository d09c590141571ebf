// k_batch.cu -- the batched path: one persistent launch for every frame of
// every cube in a batch, scheduled by data flow.
//
// A work item is (job, group, frame, PU).  Items enter a device ready queue
// only when everything they read exists: first-frame items are queued by the
// host; a frame t+1 item is queued when the CTU rows of frame t that its
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

#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

// Resident blocks per SM the register allocation aims for, per CTU size and
// block size (64 registers per thread at most where shared memory allows
// several blocks; the CTU-64 window leaves room for one).
template <int N, int NT>
constexpr int kMinBlocks = N == 64 ? 1 : (N == 32 ? (NT == 256 ? 2 : 3) : (NT == 256 ? 4 : (NT == 192 ? 5 : 6)));

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

// Rows of the previous frame read by the PUs of CTU row r.
__device__ __forceinline__ void dep_rows(int r, int N, int R, int ny, int& r0, int& r1) {
    const int lo = r * N - R - 4, hi = r * N + N - 1 + R + 4;
    r0 = lo < 0 ? 0 : lo / N;
    r1 = hi / N;
    if (r1 > ny - 1) r1 = ny - 1;
}

// Thread 0: the item at queue position `pos`, waiting (bounded) until it is
// filled.  kEmptyItem on error or timeout.
__device__ uint64_t take_item(uint64_t* queue, unsigned pos, BatchCtl* ctl) {
    uint64_t key = ld_acquire_u64(queue + pos);
    if (key != kEmptyItem) return key;
    const long long start = clock64();
    for (;;) {
        __nanosleep(64);
        key = ld_acquire_u64(queue + pos);
        if (key != kEmptyItem) return key;
        if (ld_volatile_int(&ctl->err)) return kEmptyItem;
        if (clock64() - start > ctl->budget) {
            atomicCAS(&ctl->err, 0, (int)XV_ETIMEOUT);
            return kEmptyItem;
        }
    }
}

// After the item's writes are fenced: thread 0 counts the PU in its row; if
// the row is complete, one thread per next-frame row that reads it credits
// that row's dependency counter and queues its items when the count is
// reached (the credits go out in parallel instead of one after another).
__device__ void complete_item(const JobDev& J, int job, int g, int t, int pu, uint64_t* queue, BatchCtl* ctl,
                              int* s_full) {
    const int row = pu / J.nx;
    const int64_t f = (int64_t)g * J.T + t;
    if (threadIdx.x == 0)
        *s_full = (atomicAdd(J.rowdone + f * J.ny + row, 1u) + 1u == (unsigned)J.nx) && (t + 1 < J.te);
    __syncthreads();
    if (!*s_full) return;
    const int reach = (J.R + 4 + J.ctu - 1) / J.ctu + 1;
    const int r = row - reach + (int)threadIdx.x;
    if ((int)threadIdx.x > 2 * reach || r < 0 || r >= J.ny) return;
    int r0, r1;
    dep_rows(r, J.ctu, J.R, J.ny, r0, r1);
    if (row < r0 || row > r1) return;
    const int64_t di = (f + 1) * J.ny + r;
    const unsigned need = (unsigned)(r1 - r0 + 1) + (ctl->stall_row == (long long)di && job == 0 ? 1u : 0u);
    if (atomicAdd(J.depcnt + di, 1u) + 1u == need) {
        __threadfence();
        const unsigned base = atomicAdd(&ctl->tail, (unsigned)J.nx);
        for (int i = 0; i < J.nx; ++i) {
            const uint64_t key = ((uint64_t)job << 56) | ((uint64_t)g << 48) | ((uint64_t)(t + 1) << 32) |
                                 (uint32_t)(r * J.nx + i);
            asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(queue + base + i), "l"(key) : "memory");
        }
    }
}

template <int N, int kNT>
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

template <int N, int kNT>
__global__ void __launch_bounds__(kNT, (kMinBlocks<N, kNT>))
k_persist(const JobDev* __restrict__ jobs, uint64_t* queue, BatchCtl* ctl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_pos, s_next;
    __shared__ uint64_t s_key;
    __shared__ int s_full;
    const unsigned total = ctl->total;
    if (threadIdx.x == 0) s_next = atomicAdd(&ctl->head, 1u);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned pos = s_next;
            s_pos = pos;
            s_key = pos < total ? take_item(queue, pos, ctl) : kEmptyItem;
            // take the following position now; its atomic overlaps this item
            if (pos < total) s_next = atomicAdd(&ctl->head, 1u);
        }
        __syncthreads();
        const unsigned pos = s_pos;
        const uint64_t key = s_key;
        if (pos >= total) break;
        if (key != kEmptyItem && !ld_volatile_int(&ctl->err)) {
            const int job = (int)(key >> 56);
            const JobDev& J = jobs[job];
            const int g = (int)((key >> 48) & 0xff), t = (int)((key >> 32) & 0xffff), pu = (int)(uint32_t)key;
            item_work<N, kNT>(J, g, t, pu, smem);
            __threadfence();
            __syncthreads();
            complete_item(J, job, g, t, pu, queue, ctl, &s_full);
        }
        __syncthreads();
    }
}

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
        ctl[k] = BatchCtl{0u, cls[k].nfirst, cls[k].total, 0, budget, stall_row};
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

using PersistFn = void (*)(const JobDev*, uint64_t*, BatchCtl*);
template <int NT>
PersistFn persist_fn_nt(int ctu) {
    switch (ctu) {
        case 8: return k_persist<8, NT>;
        case 16: return k_persist<16, NT>;
        case 32: return k_persist<32, NT>;
        case 64: return k_persist<64, NT>;
    }
    return nullptr;
}
PersistFn persist_fn(int ctu, int nt) {
    switch (nt) {
        case 128: return persist_fn_nt<128>(ctu);
        case 192: return persist_fn_nt<192>(ctu);
        case 256: return persist_fn_nt<256>(ctu);
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

size_t persist_smem_bytes(int ctu, int R, bool has_me) {
    size_t a = xvd::tqr_smem_bytes(ctu);
    size_t b = has_me ? xvd::me_smem_bytes(ctu, R) : 0;
    return a > b ? a : b;
}

int persist_grid(int ctu, int nt, size_t smem) {
    PersistFn fn = persist_fn(ctu, nt);
    if (!fn) return 0;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nt, smem) != cudaSuccess) {
        cudaGetLastError();  // reported by the launch that follows, not left behind
        per = 1;
    }
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_persist(int ctu, int nt, const JobDev* jobs, uint64_t* queue, BatchCtl* ctl, size_t smem,
                           int grid, cudaStream_t st) {
    PersistFn fn = persist_fn(ctu, nt);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, nt, smem, st>>>(jobs, queue, ctl);
    return cudaGetLastError();
}

}  // namespace xvh
