// Streaming (stencil-free) Krylov kernels: dot products against a basis, basis updates
// with a norm, and linear combinations.  Nodes are processed VEC at a time with 16-byte
// loads (float4 / double2) in a grid-stride loop, all loads of an iteration issued
// before any store, and the number of live accumulators fixed at compile time (NQ, the
// next power of two of the basis size) so that occupancy stays high.
#pragma once

#include <type_traits>

#include "st_device.cuh"

namespace st {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int W = 4;
    __device__ __forceinline__ static void get(const V& v, float* a) {
        a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
    }
    __device__ __forceinline__ static V make(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int W = 2;
    __device__ __forceinline__ static void get(const V& v, double* a) {
        a[0] = v.x; a[1] = v.y;
    }
    __device__ __forceinline__ static V make(const double* a) { return make_double2(a[0], a[1]); }
};

template <typename T>
__device__ __forceinline__ typename Vec16<T>::V ldv(const T* p, long long v) {
    return __ldg(reinterpret_cast<const typename Vec16<T>::V*>(p) + v);
}
template <typename T>
__device__ __forceinline__ typename Vec16<T>::V ldv_rw(const T* p, long long v) {
    return reinterpret_cast<const typename Vec16<T>::V*>(p)[v];
}
template <typename T>
__device__ __forceinline__ void stv(T* p, long long v, const T* a) {
    reinterpret_cast<typename Vec16<T>::V*>(p)[v] = Vec16<T>::make(a);
}

struct StreamCfg {
    int blocks;
};

inline __host__ int stream_blocks(long long n, int width) {
    const long long nv = (n + width - 1) / width;
    long long b = (nv + 255) / 256;
    if (b > 1216) b = 1216;  // 152 SMs x 8 resident blocks of 256 threads
    if (b < 1) b = 1;
    return (int)b;
}

// Calls f(q, lanes, nl) for each group of consecutive nodes handled by this thread: q is the
// first node, nl the number of valid nodes (W in the body, fewer in the tail).
template <typename T, typename F>
__device__ __forceinline__ void stream_loop(long long n, F&& f) {
    constexpr int W = Vec16<T>::W;
    const long long nv = n / W;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += stride) f(v, true);
    // tail: the last n % W nodes, one thread
    if (blockIdx.x == 0 && threadIdx.x == 0 && n % W) f(nv, false);
}

}  // namespace st
