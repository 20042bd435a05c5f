// Hopping-kernel instantiations for PLQ_F16 storage (18- and 12-real links).
#include "plq_hop_impl.cuh"

namespace plq {

plq_status launch_hop_f16(const HopArgs &a, int reals, int epi, cudaStream_t s, int block) {
    return reals == 12 ? dispatch_hop<PLQ_F16, 12>(a, epi, s, block) : dispatch_hop<PLQ_F16, 18>(a, epi, s, block);
}

}  // namespace plq
