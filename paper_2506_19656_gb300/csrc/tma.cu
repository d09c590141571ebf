// tma.cu -- tensor maps for the search window's TMA loads (host side).
//
// The motion search stages its reference window (channel 0 of the previous
// reconstruction) in shared memory.  Where the window lies inside the plane
// and starts 4 samples into an 8-sample chunk (the layout the search keeps:
// window column c at element y S + 4 + c), one tiled bulk copy of S x WW
// samples from chunk column xa = x0 - R - 8 brings it in: a 3-D tensor map
// over the G groups' channel-0 planes of one frame, box (S, WW, 1).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "me.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool window_map_usable(int ctu, int R) {
    const int S = xvd::me_stride(ctu, R), WW = xvd::me_win(ctu, R);
    // the window starts 4 samples into a chunk (R + 4 = 4 mod 8 for CTU-aligned
    // PUs) and the box fits the copy engine's 256-element limit
    return (R % 8) == 0 && S <= 256 && WW <= 256;
}

bool encode_window_map(WindowMap* m, const uint16_t* plane0, int Wp, int Hp, int64_t gstride, int G, int ctu, int R) {
    std::memset(m, 0, sizeof *m);
    m->polls = 1ll << 24;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !window_map_usable(ctu, R)) return false;
    if ((reinterpret_cast<uintptr_t>(plane0) & 15) || (Wp % 8) || (gstride % 8)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Wp, (cuuint64_t)Hp, (cuuint64_t)G};
    const cuuint64_t strides[2] = {(cuuint64_t)Wp * 2, (cuuint64_t)gstride * 2};
    const cuuint32_t box[3] = {(cuuint32_t)xvd::me_stride(ctu, R), (cuuint32_t)xvd::me_win(ctu, R), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(m->bytes);
    const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(plane0), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    m->valid = r == CUDA_SUCCESS ? 1 : 0;
    return m->valid != 0;
}

}  // namespace xvh
