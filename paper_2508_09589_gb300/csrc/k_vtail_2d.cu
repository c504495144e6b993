// Persistent coarse V-cycle tail, 2-D space, double multigrid (see k_vtail.cuh).
#include "k_vtail.cuh"

namespace st {
template int launch_vtail_sd<2, double>(bool, const VTail<double>*, unsigned*, cudaStream_t);
}  // namespace st
