// Device-side building blocks: Dirichlet masks, the level-0 matrix-free element
// rows, the coarse element-block rows, and a deterministic grid reduction.
#pragma once

#include <type_traits>

#include "st_internal.h"

namespace st {

// ---------------------------------------------------------------- masks
// Spatial part of the prescribed set: the sink patch on the x = 0 (or y = 0) face,
// all walls, or nothing.  The whole t = 0 plane is prescribed as the initial condition.
template <int SD>
__device__ __forceinline__ bool sp_dir(const Geom& g, int i, int j, int k) {
    if (g.bc == ST_BC_NONE) return false;
    if (g.bc == ST_BC_ALL_WALLS) {
        bool w = i == 0 || i == g.nx1 - 1 || j == 0 || j == g.ny1 - 1;
        if (SD == 3) w = w || k == 0 || k == g.nz1 - 1;
        return w;
    }
    const int idx[3] = {i, j, k};
    if (idx[g.face] != 0) return false;
#pragma unroll
    for (int d = 0; d < SD; ++d)
        if (d != g.face && (idx[d] < g.plo[d] || idx[d] > g.phi[d])) return false;
    return true;
}

template <int SD>
__device__ __forceinline__ bool is_free(const Geom& g, int i, int j, int k, int n) {
    return n > 0 && !sp_dir<SD>(g, i, j, k);
}

template <typename T>
__device__ __forceinline__ T ipow(T x, int p) {
    T r = T(1);
    for (int q = 0; q < p; ++q) r *= x;
    return r;
}

template <int NS>
__host__ __device__ constexpr int symidx(int i, int j) {
    return i <= j ? i * NS - i * (i - 1) / 2 + (j - i) : j * NS - j * (j - 1) / 2 + (i - j);
}

// ---------------------------------------------------------------- loaders
template <typename T, typename TX>
struct LoadPlain {
    const TX* __restrict__ x;
    __device__ __forceinline__ T operator()(long long q) const { return (T)x[q]; }
};

// x_q = d_q u_q (right Jacobi preconditioning inside the smoother)
template <typename T>
struct LoadScaled {
    const T* __restrict__ u;
    const T* __restrict__ d;
    __device__ __forceinline__ T operator()(long long q) const { return u[q] * d[q]; }
};

// ---------------------------------------------------------------- level 0 (matrix free)
template <typename T>
__device__ __forceinline__ void coef_l0(const OpL0<T>& op, long long e, T& C, T& k) {
    T gm;
    if constexpr (std::is_same<T, float>::value)
        gm = __bfloat162float(op.g16[e]);
    else
        gm = op.g64[e];
    C = (T)op.simp.C_ins + (T)op.simp.dC * ipow(gm, op.simp.p_c);
    k = (T)op.simp.k_ins + (T)op.simp.dk * ipow(gm, op.simp.p_k);
}

// Row of the level-0 operator at a free node (i, j, k, n): the sum over the adjacent
// elements of row a of C_e (D_t (x) M_x) + k_e (M_t (x) K_x), with D_t = [[0,0],[-1,1]]
// (upwind in time) and M_t = dt/6 [[2,1],[1,2]]; prescribed neighbours contribute 0.
// TR selects the transposed operator (column a instead of row a).
template <int SD, typename T, bool TR, typename L>
__device__ __forceinline__ T row_l0(const OpL0<T>& op, int i, int j, int k, int n, const L& ld) {
    const Geom& g = op.g;
    constexpr int NS = 1 << SD;
    const long long P = g.plane;
    const bool below = n > 0, above = n < g.net;
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1);
        const int ez = (SD == 3) ? k - 1 + ((o >> 2) & 1) : 0;
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
        if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
        const int as = (~o) & (NS - 1);
        const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
        T Cb = 0, kb = 0, Ca = 0, ka = 0;
        if (below) coef_l0(op, op.tc ? se : (long long)(n - 1) * g.sp_elems + se, Cb, kb);
        if (above) {
            if (op.tc && below) {
                Ca = Cb;
                ka = kb;
            } else {
                coef_l0(op, op.tc ? se : (long long)n * g.sp_elems + se, Ca, ka);
            }
        }
#pragma unroll
        for (int bs = 0; bs < NS; ++bs) {
            const int ni = ex + (bs & 1), nj = ey + ((bs >> 1) & 1);
            const int nk = (SD == 3) ? ez + ((bs >> 2) & 1) : 0;
            T xm = 0, x0 = 0, xp = 0;
            if (!sp_dir<SD>(g, ni, nj, nk)) {
                const long long sidx = ((long long)nk * g.ny1 + nj) * g.nx1 + ni;
                if (n - 1 > 0) xm = ld((long long)(n - 1) * P + sidx);
                if (n > 0) x0 = ld((long long)n * P + sidx);
                if (above) xp = ld((long long)(n + 1) * P + sidx);
            }
            const T m = op.mxd[as ^ bs], kk = op.kxd[as ^ bs];
            if (below) acc += Cb * m * (TR ? x0 : (x0 - xm)) + kb * kk * op.dt6 * (xm + T(2) * x0);
            if (above) {
                if (TR) acc -= Ca * m * xp;
                acc += ka * kk * op.dt6 * (T(2) * x0 + xp);
            }
        }
    }
    return acc;
}

template <int SD, typename T>
__device__ __forceinline__ T diag_l0(const OpL0<T>& op, int i, int j, int k, int n) {
    const Geom& g = op.g;
    constexpr int NS = 1 << SD;
    const bool below = n > 0, above = n < g.net;
    T acc = 0;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1);
        const int ez = (SD == 3) ? k - 1 + ((o >> 2) & 1) : 0;
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
        if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
        const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
        T C, kk;
        if (below) {
            coef_l0(op, op.tc ? se : (long long)(n - 1) * g.sp_elems + se, C, kk);
            acc += C * op.mxd[0] + kk * op.kxd[0] * T(2) * op.dt6;
        }
        if (above) {
            coef_l0(op, op.tc ? se : (long long)n * g.sp_elems + se, C, kk);
            acc += kk * op.kxd[0] * T(2) * op.dt6;
        }
    }
    return acc;
}

// ---------------------------------------------------------------- coarse levels (element blocks)
template <typename T>
__device__ __forceinline__ long long elem_index(const OpLc<T>& op, int slab, long long se) {
    return op.tc ? ((slab == 0 ? 0 : 1) * op.g.sp_elems + se) : ((long long)slab * op.g.sp_elems + se);
}

template <int SD, typename T, bool TR, typename L>
__device__ __forceinline__ T row_lc(const OpLc<T>& op, int i, int j, int k, int n, const L& ld) {
    const Geom& g = op.g;
    constexpr int NS = 1 << SD, NSYM = NS * (NS + 1) / 2, NV = 4 * NSYM;
    const long long P = g.plane;
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1);
        const int ez = (SD == 3) ? k - 1 + ((o >> 2) & 1) : 0;
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
        if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
        const int as = (~o) & (NS - 1);
        const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
#pragma unroll
        for (int sb = 0; sb < 2; ++sb) {
            const int slab = n - 1 + sb;
            if (slab < 0 || slab >= g.net) continue;
            const int at = 1 - sb;
            const T* A = op.elem + elem_index(op, slab, se) * NV;
#pragma unroll
            for (int bt = 0; bt < 2; ++bt) {
                const long long pl = (long long)(slab + bt) * P;
                const int blk = TR ? (bt * 2 + at) : (at * 2 + bt);
#pragma unroll
                for (int bs = 0; bs < NS; ++bs) {
                    const int ni = ex + (bs & 1), nj = ey + ((bs >> 1) & 1);
                    const int nk = (SD == 3) ? ez + ((bs >> 2) & 1) : 0;
                    const long long sidx = ((long long)nk * g.ny1 + nj) * g.nx1 + ni;
                    acc += A[blk * NSYM + symidx<NS>(as, bs)] * ld(pl + sidx);
                }
            }
        }
    }
    return acc;
}

template <int SD, typename T>
__device__ __forceinline__ T diag_lc(const OpLc<T>& op, int i, int j, int k, int n) {
    const Geom& g = op.g;
    constexpr int NS = 1 << SD, NSYM = NS * (NS + 1) / 2, NV = 4 * NSYM;
    T acc = 0;
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1);
        const int ez = (SD == 3) ? k - 1 + ((o >> 2) & 1) : 0;
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
        if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
        const int as = (~o) & (NS - 1);
        const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
        for (int sb = 0; sb < 2; ++sb) {
            const int slab = n - 1 + sb;
            if (slab < 0 || slab >= g.net) continue;
            const int at = 1 - sb;
            const T* A = op.elem + elem_index(op, slab, se) * NV;
            acc += A[(at * 2 + at) * NSYM + symidx<NS>(as, as)];
        }
    }
    return acc;
}

// Level-generic row: LV = 0 (matrix free) or 1 (element blocks).
template <int SD, typename T, int LV, bool TR, typename L>
__device__ __forceinline__ T op_row(const OpL0<T>& o0, const OpLc<T>& oc, int i, int j, int k, int n,
                                    const L& ld) {
    if constexpr (LV == 0)
        return row_l0<SD, T, TR>(o0, i, j, k, n, ld);
    else
        return row_lc<SD, T, TR>(oc, i, j, k, n, ld);
}

// ---------------------------------------------------------------- node iteration
// Grid: block (32, 8) over (i, j); blockIdx.z strides over the nz1 * nt1 planes.
#define ST_NODE_LOOP_BEGIN(G)                                                  \
    const int i_ = blockIdx.x * blockDim.x + threadIdx.x;                      \
    const int j_ = blockIdx.y * blockDim.y + threadIdx.y;                      \
    const bool inplane_ = i_ < (G).nx1 && j_ < (G).ny1;                        \
    for (int z_ = blockIdx.z; z_ < (G).nz1 * (G).nt1; z_ += gridDim.z) {       \
        const int n_ = z_ / (G).nz1, k_ = z_ - n_ * (G).nz1;                   \
        const long long idx_ = ((long long)z_ * (G).ny1 + j_) * (G).nx1 + i_; \
        if (inplane_) {
#define ST_NODE_LOOP_END \
    }                    \
    }

// ---------------------------------------------------------------- deterministic reduction
// Every block publishes nq partial sums; the last block to finish sums them in block
// order (independent of which block finished last) into `out` (shared memory of the
// last block).  Returns true in the last block, after a __syncthreads().
template <int NQ>
__device__ __forceinline__ bool reduce_publish(const double (&v)[NQ], int nq, RedBuf rb, double* out) {
    __shared__ double sm_[NQ][32];
    __shared__ int last_;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q < nq) {
            double a = v[q];
#pragma unroll
            for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
            if (lane == 0) sm_[q][warp] = a;
        }
    }
    __syncthreads();
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    if (tid < nq) {
        double a = 0;
        for (int w = 0; w < nw; ++w) a += sm_[tid][w];
        rb.part[bid * kRedQ + tid] = a;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned t = atomicAdd(rb.counter, 1u);
        last_ = (t == (unsigned)(nb - 1));
    }
    __syncthreads();
    if (!last_) return false;
    __threadfence();
    for (int q = warp; q < nq; q += nw) {
        double a = 0;
        for (long long b = lane; b < nb; b += 32) a += __ldcg(rb.part + b * kRedQ + q);
#pragma unroll
        for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) out[q] = a;
    }
    if (tid == 0) *rb.counter = 0u;
    __syncthreads();
    return true;
}

}  // namespace st
