// k_batch_ctu8.cu -- the persistent kernel for 8x8 CTUs, all block sizes.
#include "batch.cuh"

namespace xvh {
batch::PersistFn persist_fn_ctu8(int nt, bool decode) { return batch::persist_fn_for<8>(nt, decode); }
}  // namespace xvh
