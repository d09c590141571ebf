// k_batch_ctu16.cu -- the persistent kernel for 16x16 CTUs, all block sizes.
#include "batch.cuh"

namespace xvh {
batch::PersistFn persist_fn_ctu16(int nt, bool decode) { return batch::persist_fn_for<16>(nt, decode); }
}  // namespace xvh
