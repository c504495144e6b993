// float instantiation of the fused smoother step kernel (k_smstep.cuh).
#include "k_smstep.cuh"

namespace st {
template void launch_sm_step<float>(const Geom&, const float*, const float*, const unsigned char*, const float*,
                                   const Ptrs<float>&, const float*, float*, int, int, SmState*, RedBuf, cudaStream_t);
template bool sm_step_aligned<float>(const Ptrs<float>&, int, const float*, const float*, long long, long long);
}  // namespace st
