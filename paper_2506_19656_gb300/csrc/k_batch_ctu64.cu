// k_batch_ctu64.cu -- the persistent kernel for 64x64 CTUs, all block sizes.
#include "batch.cuh"

namespace xvh {
batch::PersistFn persist_fn_ctu64(int nt, bool decode) { return batch::persist_fn_for<64>(nt, decode); }
}  // namespace xvh
