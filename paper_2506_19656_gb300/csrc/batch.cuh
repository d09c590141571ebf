// batch.cuh -- the persistent data-flow kernel of the batched path (device
// code; instantiated per CTU size in k_batch_ctu*.cu).  See k_batch.cu for
// the scheduling scheme.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "dec.cuh"
#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

namespace xvh {
namespace batch {

using PersistFn = void (*)(const JobDev*, uint64_t*, BatchCtl*);

namespace {  // each including file gets its own copies


// Resident blocks per SM the register allocation aims for, per CTU size and
// block size (64 to 128 registers per thread where shared memory allows
// several blocks; the CTU-64 window leaves room for one).  Measured: CTU 16
// at 128 threads is fastest with six (seven spill nothing at 72 registers
// but run slower), CTU 32 at 128 threads with four (128 registers, no
// spills) rather than three.
template <int N, int NT>
constexpr int kMinBlocks = NT == 512 ? (N == 64 ? 1 : 2)
                                     : N == 64 ? 1 : (N == 32 ? (NT == 256 ? 2 : 3) : (NT == 256 ? 4 : (NT == 192 ? 5 : 6)));

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

// Encodes (kDecode: decodes) one PU; returns the integer-search candidates
// evaluated exactly.  Decoding is a separate instantiation so that the
// encoder's code carries none of it (smaller code, fewer spills).
template <int N, int kNT, bool kDecode>
__device__ uint32_t item_work(const JobDev& J, int g, int t, int pu, unsigned char* smem) {
    const int64_t plane = (int64_t)J.Hp * J.Wp, fsz = 3 * plane;
    const int64_t f = (int64_t)g * J.T + t;
    const uint16_t* ref = t > 0 ? J.recon + (f - 1) * fsz : nullptr;
    const int x0 = (pu % J.nx) * N, y0 = (pu / J.nx) * N;
    if constexpr (kDecode) {
        const int64_t o = f * (int64_t)J.nx * J.ny + pu;
        const int mvx = ref ? J.mv[2 * o] : 0, mvy = ref ? J.mv[2 * o + 1] : 0;
        const uint32_t b = xvd::dec_cu<N, kNT, true>(J.levels + f * fsz, ref, plane, J.Hp, J.Wp, x0, y0, mvx, mvy,
                                                     J.tu[o], J.qp, J.recon + f * fsz, smem);
        if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(J.bits + f), (unsigned long long)b);
        return 0u;
    } else {
        const uint16_t* cur = J.planes + f * fsz;
        xvd::MeResult m{0, 0, 0u, 0, 0, 0u, 0u};
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
        return m.exact_cand;
    }
}

template <int N, int kNT, bool kDecode>
__global__ void __launch_bounds__(kNT, (kMinBlocks<N, kNT>))
k_persist(const JobDev* __restrict__ jobs, uint64_t* queue, BatchCtl* ctl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_pos, s_next;
    __shared__ uint64_t s_key;
    __shared__ int s_full;
    const unsigned total = ctl->total;
    unsigned long long exact = 0;  // thread 0: this block's exactly evaluated candidates
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
            exact += item_work<N, kNT, kDecode>(J, g, t, pu, smem);
            __threadfence();
            __syncthreads();
            complete_item(J, job, g, t, pu, queue, ctl, &s_full);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && exact) atomicAdd(&ctl->exact_cand, exact);
}


template <int N, bool kDecode>
PersistFn persist_fn_nt(int nt) {
    switch (nt) {
        case 128: return k_persist<N, 128, kDecode>;
        case 192: return k_persist<N, 192, kDecode>;
        case 256: return k_persist<N, 256, kDecode>;
        case 512: return k_persist<N, 512, kDecode>;
    }
    return nullptr;
}

template <int N>
PersistFn persist_fn_for(int nt, bool decode) {
    return decode ? persist_fn_nt<N, true>(nt) : persist_fn_nt<N, false>(nt);
}

}  // namespace
}  // namespace batch
}  // namespace xvh
