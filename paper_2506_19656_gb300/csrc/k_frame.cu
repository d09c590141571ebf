// k_frame.cu -- the plain path's per-frame kernels: one thread block per PU
// for motion estimation, one per CU for transform/quantise/reconstruct, all
// groups of the frame in one launch (grid.y = group).
#include <cuda_runtime.h>

#include <cstdint>

#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

// Threads per block and the resident blocks per SM the register allocation
// aims for.  CTU 32: the search at 128 threads x 6 blocks (six 34 KB
// windows fit the SM's shared memory) and the transform at 192 threads x 4
// blocks, one warp per channel half-CU (tqr_cu_w32); both measured faster
// than 256 threads x 3 blocks, results unchanged.  CTU 64: the search and the
// transform at 512 threads (one block per SM either way; the search 9 %
// faster than at 256).
template <int N> constexpr int kNTMe = N == 32 ? 128 : (N == 64 ? 512 : 256);
template <int N> constexpr int kNTTqr = N == 32 ? 192 : (N == 64 ? 512 : 256);
template <int N> constexpr int kMinBlocksMe = N == 64 ? 1 : (N == 32 ? 6 : 4);
template <int N> constexpr int kMinBlocksTqr = N == 64 ? 1 : 4;

template <int N, int KC>
__global__ void __launch_bounds__(kNTMe<N>, kMinBlocksMe<N>)
k_me_frame(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, int64_t gstride, int Hp, int Wp,
           int R, int64_t lmv, int16_t* mv, uint32_t* cost, int16_t* mv_int, uint32_t* cost_int,
           int64_t pu_gstride, unsigned long long* exact, const __grid_constant__ WindowMap wmap, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int pu = blockIdx.x, g = blockIdx.y, nx = Wp / N;
    xvd::MeResult r = xvd::me_pu<N, kNTMe<N>, false, KC>(cur + g * gstride, ref + g * gstride, Hp, Wp, (pu % nx) * N,
                                         (pu / nx) * N, R, lmv, smem, wmap.valid ? wmap.bytes : nullptr, g, err,
                                         wmap.polls);
    if (threadIdx.x == 0) {
        const int64_t o = g * pu_gstride + pu;
        mv[2 * o] = (int16_t)r.mvx;
        mv[2 * o + 1] = (int16_t)r.mvy;
        if (cost) cost[o] = r.cost;
        if (mv_int) { mv_int[2 * o] = (int16_t)r.mvx_int; mv_int[2 * o + 1] = (int16_t)r.mvy_int; }
        if (cost_int) cost_int[o] = r.cost_int;
        if (exact) atomicAdd(exact, (unsigned long long)r.exact_cand);
    }
}

template <int N>
__global__ void __launch_bounds__(kNTTqr<N>, kMinBlocksTqr<N>)
k_tqr_frame(const uint16_t* __restrict__ cur, const uint16_t* __restrict__ ref, const int16_t* __restrict__ mv,
            int64_t gstride, int Hp, int Wp, int qp, unsigned tu_mask, int64_t lf8, int64_t pu_gstride,
            uint16_t* recon, int16_t* levels, uint8_t* tu_log2, uint64_t* bits, int64_t bits_gstride) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int cu = blockIdx.x, g = blockIdx.y, nx = Wp / N;
    const int64_t o = g * pu_gstride + cu;
    int mvx = 0, mvy = 0;
    if (ref) { mvx = mv[2 * o]; mvy = mv[2 * o + 1]; }
    uint32_t b = xvd::tqr_cu<N, kNTTqr<N>>(cur + g * gstride, ref ? ref + g * gstride : nullptr, (int64_t)Hp * Wp, Hp,
                                     Wp, (cu % nx) * N, (cu / nx) * N, mvx, mvy, qp, tu_mask, lf8,
                                     recon + g * gstride, levels ? levels + g * gstride : nullptr,
                                     tu_log2 ? tu_log2 + o : nullptr, smem);
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(bits + g * bits_gstride),
                                    (unsigned long long)b);
}

template <int N, int KC>
cudaError_t me_nk(const uint16_t* cur, const uint16_t* ref, int G, int64_t gstride, int Hp, int Wp,
                  const xv_params* p, int16_t* mv, uint32_t* cost, int16_t* mv_int, uint32_t* cost_int,
                  int64_t pu_gstride, cudaStream_t st, unsigned long long* exact, const WindowMap* wmap, int* err) {
    WindowMap m{};
    if (wmap && wmap->valid && err) m = *wmap;
    size_t smem = xvd::me_smem_bytes(N, p->search_range, KC);
    cudaError_t e = cudaFuncSetAttribute(k_me_frame<N, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((Hp / N) * (Wp / N), G);
    k_me_frame<N, KC><<<grid, kNTMe<N>, smem, st>>>(cur, ref, gstride, Hp, Wp, p->search_range, p->lambda_mv_fp16, mv,
                                                    cost, mv_int, cost_int, pu_gstride, exact, m, err);
    return cudaGetLastError();
}

// CTU 16: the whole box table at once (one class) where the search's shared
// memory still leaves its four blocks per SM (measured on DeepExtremeCubes-
// sized frames: 0.026 -> 0.021 ms per launch), else four row classes.
template <int N>
cudaError_t me_n(const uint16_t* cur, const uint16_t* ref, int G, int64_t gstride, int Hp, int Wp,
                 const xv_params* p, int16_t* mv, uint32_t* cost, int16_t* mv_int, uint32_t* cost_int,
                 int64_t pu_gstride, cudaStream_t st, unsigned long long* exact, const WindowMap* wmap, int* err) {
    if constexpr (N == 16) {
        if (xvd::me_smem_bytes(N, p->search_range, 1) <= 56 * 1024)
            return me_nk<N, 1>(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride, st, exact,
                               wmap, err);
    }
    return me_nk<N, xvd::me_kcls(N)>(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride, st,
                                     exact, wmap, err);
}

template <int N>
cudaError_t tqr_n(const uint16_t* cur, const uint16_t* ref, const int16_t* mv, int G, int64_t gstride, int Hp,
                  int Wp, const xv_params* p, int64_t pu_gstride, uint16_t* recon, int16_t* levels,
                  uint8_t* tu_log2, uint64_t* bits, int64_t bits_gstride, cudaStream_t st) {
    const size_t smem = N == 32 && kNTTqr<N> == xvd::kW32Threads ? xvd::tqr_w32_smem_bytes() : xvd::tqr_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(k_tqr_frame<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((Hp / N) * (Wp / N), G);
    k_tqr_frame<N><<<grid, kNTTqr<N>, smem, st>>>(cur, ref, mv, gstride, Hp, Wp, p->qp, p->tu_mask, p->lambda_fp8,
                                            pu_gstride, recon, levels, tu_log2, bits, bits_gstride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_me_frame(const uint16_t* cur, const uint16_t* ref, int G, int64_t gstride, int Hp, int Wp,
                            const xv_params* p, int16_t* mv, uint32_t* cost, int16_t* mv_int,
                            uint32_t* cost_int, int64_t pu_gstride, cudaStream_t st, unsigned long long* exact,
                            const WindowMap* wmap, int* err) {
    switch (p->ctu) {
        case 8: return me_n<8>(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride, st, exact, wmap, err);
        case 16: return me_n<16>(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride, st, exact, wmap, err);
        case 32: return me_n<32>(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride, st, exact, wmap, err);
        case 64: return me_n<64>(cur, ref, G, gstride, Hp, Wp, p, mv, cost, mv_int, cost_int, pu_gstride, st, exact, wmap, err);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tqr_frame(const uint16_t* cur, const uint16_t* ref, const int16_t* mv, int G, int64_t gstride,
                             int Hp, int Wp, const xv_params* p, int64_t pu_gstride, uint16_t* recon,
                             int16_t* levels, uint8_t* tu_log2, uint64_t* bits, int64_t bits_gstride,
                             cudaStream_t st) {
    switch (p->ctu) {
        case 8: return tqr_n<8>(cur, ref, mv, G, gstride, Hp, Wp, p, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st);
        case 16: return tqr_n<16>(cur, ref, mv, G, gstride, Hp, Wp, p, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st);
        case 32: return tqr_n<32>(cur, ref, mv, G, gstride, Hp, Wp, p, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st);
        case 64: return tqr_n<64>(cur, ref, mv, G, gstride, Hp, Wp, p, pu_gstride, recon, levels, tu_log2, bits, bits_gstride, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace xvh
