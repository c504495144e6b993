// Persistent coarse V-cycle tail, 2-D space, float multigrid (see k_vtail.cuh).
#include "k_vtail.cuh"

namespace st {
template int launch_vtail_sd<2, float>(bool, const VTail<float>*, unsigned*, cudaStream_t);
}  // namespace st
