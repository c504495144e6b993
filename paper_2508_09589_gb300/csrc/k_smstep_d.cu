// double instantiation of the fused smoother step kernel (k_smstep.cuh).
#include "k_smstep.cuh"

namespace st {
template void launch_sm_step<double>(const Geom&, const double*, const double*, const unsigned char*, const double*,
                                   const Ptrs<double>&, const double*, double*, int, int, SmState*, RedBuf, cudaStream_t);
template bool sm_step_aligned<double>(const Ptrs<double>&, int, const double*, const double*, long long, long long);
}  // namespace st
