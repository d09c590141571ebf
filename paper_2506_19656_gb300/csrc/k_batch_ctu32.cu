// k_batch_ctu32.cu -- the persistent kernel for 32x32 CTUs, all block sizes.
#include "batch.cuh"

namespace xvh {
batch::PersistFn persist_fn_ctu32(int nt, bool decode) { return batch::persist_fn_for<32>(nt, decode); }
}  // namespace xvh
