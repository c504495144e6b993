#pragma once
// Shared-memory staging helpers of the time-marching ring kernels: 16-byte cp.async chunk
// copies into the dynamic shared memory, and plain loads and stores into it by byte offset.
#include <stdint.h>

#include "st_device.cuh"

namespace st {

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using V = float2;
};
template <>
struct Pair<double> {
    using V = double2;
};

__device__ __forceinline__ void cp_async16(unsigned smem_dst, const void* gsrc, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_dst), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}

// The ring kernels' dynamic shared memory, and plain loads and stores into it by byte offset
// (32-bit shared addressing; the compiler may reorder and interleave them, while cp.async and
// barriers keep their places).
extern __shared__ __align__(16) unsigned char g_step_smem[];
template <typename T>
__device__ __forceinline__ T lds1(unsigned a) {
    return *reinterpret_cast<const T*>(g_step_smem + a);
}
template <typename T>
__device__ __forceinline__ void lds2(unsigned a, T& x, T& y) {
    const typename Pair<T>::V v = *reinterpret_cast<const typename Pair<T>::V*>(g_step_smem + a);
    x = v.x;
    y = v.y;
}
template <typename T>
__device__ __forceinline__ void sts2(unsigned a, T x, T y) {
    typename Pair<T>::V v;
    v.x = x;
    v.y = y;
    *reinterpret_cast<typename Pair<T>::V*>(g_step_smem + a) = v;
}

}  // namespace st
