// Persistent batched CG kernel, inner precision F32 with 12-real links (one
// translation unit per inner format, compiled in parallel).
#include "plq_batched_impl.cuh"

namespace plq {
namespace batch {

plq_status launch_f32_12(const BatchArgs &a, int shape, int bps, cudaStream_t s, Ctx::BatchCache &c, LaunchOut *o) {
    return launch_batched<PLQ_F32, 12>(a, shape, bps, s, c, o);
}

}  // namespace batch
}  // namespace plq
