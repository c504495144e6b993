// Persistent coarse V-cycle tail, 3-D space, float multigrid (see k_vtail.cuh).
#include "k_vtail.cuh"

namespace st {
template int launch_vtail_sd<3, float>(bool, const VTail<float>*, unsigned*, cudaStream_t);
}  // namespace st
