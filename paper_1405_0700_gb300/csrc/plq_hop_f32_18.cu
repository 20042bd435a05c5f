// Hopping-kernel instantiations for PLQ_F32 storage, 18-real links.
#include "plq_hop_impl.cuh"

namespace plq {

plq_status launch_hop_f32_18(const HopArgs &a, int epi, cudaStream_t s, int block) {
    return dispatch_hop<PLQ_F32, 18>(a, epi, s, block);
}

}  // namespace plq
