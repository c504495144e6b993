// Descriptor of the persistent coarse tail of the V-cycle (k_vtail.cuh, instantiated in k_vtail_*.cu), kept in device memory.
#pragma once

#include "st_internal.h"

namespace st {

template <typename T>
struct VLevel {
    Geom g;
    int lv;                        // level index (0 = fine)
    int to_next;                   // transfer to the next level: 0 space, 1 time, 2 both, -1 coarsest
    int tc;                        // extruded design (2 element versions per spatial element)
    const T* coef[2];              // 27-point stencils (extruded, 2-D) for each orientation, or null
    const unsigned char* dir;
    const T* elem;                 // element blocks (levels >= 1)
    T* b;
    T* x;
    T* r;
    T* w;
    const T* dinv;
    T* U[kMaxSmooth + 1];
};

template <typename T>
struct VTail {
    int first;                     // first level run by the kernel
    int L;                         // number of levels
    int steps;                     // smoothing steps
    int nc;                        // coarsest node count
    const double* Ainv;            // coarsest inverse (row-major)
    double* part;                  // 2 x kMaxBlocks x kRedQ partial sums
    unsigned* bar;                 // grid barrier counter (zeroed before each launch)
    int* err;                      // set on a barrier timeout
    unsigned long long* trace;     // optional: block 0 records %globaltimer after each barrier
    int trace_cap;
    unsigned spin_limit;           // polls before a grid-barrier wait gives up (default 2^24)
    OpL0<T> op0;                   // level-0 operator (when first == 0)
    VLevel<T> lv[kMaxLevels];
};

template <int SD, typename T>
int launch_vtail_sd(bool tr, const VTail<T>* dev_pv, unsigned* bar, cudaStream_t s);
template <typename T>
inline int launch_vtail(int sd, bool tr, const VTail<T>* dev_pv, unsigned* bar, cudaStream_t s) {
    return sd == 2 ? launch_vtail_sd<2, T>(tr, dev_pv, bar, s) : launch_vtail_sd<3, T>(tr, dev_pv, bar, s);
}

}  // namespace st

#define ST_SD_DISPATCH2(sd, ...)  \
    do {                          \
        if ((sd) == 2) {          \
            constexpr int SD = 2; \
            __VA_ARGS__;          \
        } else {                  \
            constexpr int SD = 3; \
            __VA_ARGS__;          \
        }                         \
    } while (0)
