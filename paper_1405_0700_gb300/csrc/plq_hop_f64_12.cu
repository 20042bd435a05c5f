// Hopping-kernel instantiations for PLQ_F64 storage, 12-real links.
#include "plq_hop_impl.cuh"

namespace plq {

plq_status launch_hop_f64_12(const HopArgs &a, int epi, cudaStream_t s, int block) {
    return dispatch_hop<PLQ_F64, 12>(a, epi, s, block);
}

}  // namespace plq
