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
// Loaders give the operator input at node q.  The raw interface (NR raw values of type R,
// combined later) lets the time-marching kernels prefetch loads without consuming them.
template <typename T, typename TX>
struct LoadPlain {
    const TX* __restrict__ x;
    using R = TX;
    static constexpr int NR = 1;
    __device__ __forceinline__ T operator()(long long q) const { return (T)x[q]; }
    __device__ __forceinline__ void raw(long long q, R* r) const { r[0] = x[q]; }
    __device__ __forceinline__ static T combine(const R* r) { return (T)r[0]; }
};

// x_q = d_q u_q (right Jacobi preconditioning inside the smoother)
template <typename T>
struct LoadScaled {
    const T* __restrict__ u;
    const T* __restrict__ d;
    using R = T;
    static constexpr int NR = 2;
    __device__ __forceinline__ T operator()(long long q) const { return u[q] * d[q]; }
    __device__ __forceinline__ void raw(long long q, R* r) const {
        r[0] = u[q];
        r[1] = d[q];
    }
    __device__ __forceinline__ static T combine(const R* r) { return r[0] * r[1]; }
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

// Sum of partials part[b * kRedQ + q] over b < nb by one warp, in a fixed order: each lane
// adds its strided share with 16 loads in flight per round, then a shuffle tree.  TA is
// the accumulation type: float in the FP32 multigrid (FP64 arithmetic is a slow path on
// this GPU, a few FMAs per clock per SM), double in the FP64 Krylov solver.
template <typename TA>
__device__ __forceinline__ void out_sum_partials_t(const TA* part, long long nb, int q, int lane, double* out) {
    TA acc[4] = {TA(0), TA(0), TA(0), TA(0)};
    for (long long b0 = lane; b0 < nb; b0 += 32 * 16) {
        TA v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const long long b = b0 + 32LL * u;
            v[u] = b < nb ? __ldcg(part + b * kRedQ + q) : TA(0);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u & 3] += v[u];
    }
    TA a = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) out[q] = (double)a;
}

__device__ __forceinline__ void out_sum_partials(const double* part, long long nb, int q, int lane, double* out) {
    out_sum_partials_t<double>(part, nb, q, lane, out);
}

// ---------------------------------------------------------------- deterministic reduction
// Every block publishes nq partial sums; the last block to finish sums them in block
// order (independent of which block finished last) into `out` (shared memory of the
// last block).  Returns true in the last block, after a __syncthreads().
template <typename TA, int NQ>
__device__ __forceinline__ bool reduce_publish_t(const TA (&v)[NQ], int nq, RedBuf rb, double* out) {
    __shared__ TA sm_[NQ][32];
    __shared__ int last_;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    TA* part = reinterpret_cast<TA*>(rb.part);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q < nq) {
            TA a = v[q];
#pragma unroll
            for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
            if (lane == 0) sm_[q][warp] = a;
        }
    }
    __syncthreads();
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    if (tid < nq) {
        TA a = 0;
        for (int w = 0; w < nw; ++w) a += sm_[tid][w];
        part[bid * kRedQ + tid] = a;
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
    for (int q = warp; q < nq; q += nw) out_sum_partials_t<TA>(part, nb, q, lane, out);
    if (tid == 0) *rb.counter = 0u;
    __syncthreads();
    return true;
}

template <int NQ>
__device__ __forceinline__ bool reduce_publish(const double (&v)[NQ], int nq, RedBuf rb, double* out) {
    return reduce_publish_t<double, NQ>(v, nq, rb, out);
}

}  // namespace st

namespace st {

// ---------------------------------------------------------------- element blocks
// Masked element matrix of element (slab, spatial ex, ey, ez) in block form:
// F[a_t * 2 + b_t][sym(a_s, b_s)], rows and columns of prescribed nodes zeroed.
template <int SD>
__device__ void l0_blocks(const OpL0<double>& op, int slab, int ex, int ey, int ez, double* F) {
    constexpr int NS = 1 << SD, NSYM = NS * (NS + 1) / 2;
    const Geom& g = op.g;
    const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
    double C, k;
    coef_l0(op, op.tc ? se : (long long)slab * g.sp_elems + se, C, k);
    bool fr[2 * NS];
    for (int at = 0; at < 2; ++at)
        for (int as = 0; as < NS; ++as)
            fr[at * NS + as] = (slab + at > 0) &&
                               !sp_dir<SD>(g, ex + (as & 1), ey + ((as >> 1) & 1), SD == 3 ? ez + ((as >> 2) & 1) : 0);
    const double Dt[2][2] = {{0.0, 0.0}, {-1.0, 1.0}};
    const double Mt[2][2] = {{2.0 * op.dt6, op.dt6}, {op.dt6, 2.0 * op.dt6}};
    for (int at = 0; at < 2; ++at)
        for (int bt = 0; bt < 2; ++bt)
            for (int as = 0; as < NS; ++as)
                for (int bs = as; bs < NS; ++bs) {
                    const double v = C * Dt[at][bt] * op.mxd[as ^ bs] + k * Mt[at][bt] * op.kxd[as ^ bs];
                    const bool m = fr[at * NS + as] && fr[bt * NS + bs];
                    F[(at * 2 + bt) * NSYM + symidx<NS>(as, bs)] = m ? v : 0.0;
                }
}

// Interpolation weight of coarse local node b (0|1) at fine position r (0, 1, 2) along a
// halved axis: r = 0 -> (1, 0), r = 1 -> (1/2, 1/2), r = 2 -> (0, 1).
inline __device__ double q1(int r, int b) {
    return r == 1 ? 0.5 : ((r == 0) == (b == 0) ? 1.0 : 0.0);
}

// ---------------------------------------------------------------- transfers (per node)
// kind: 0 = space (all spatial axes halved), 1 = time, 2 = both.
// Restriction r_c = D_c P^T D_f r_f at coarse node (i, j, k, n); P trilinear, vertex nested.
template <int SD, typename T>
__device__ __forceinline__ T restrict_node(const Geom& gf, const Geom& gc, int kind, const T* __restrict__ rf, int i,
                                           int j, int k, int n) {
    if (!is_free<SD>(gc, i, j, k, n)) return T(0);
    const bool cs = kind != 1, ct = kind != 0;
    const int I = cs ? 2 * i : i, J = cs ? 2 * j : j, K = (cs && SD == 3) ? 2 * k : k;
    const int N = ct ? 2 * n : n;
    const int rs = cs ? 1 : 0, rt = ct ? 1 : 0, rz = (cs && SD == 3) ? 1 : 0;
    T acc = 0;
    for (int dn = -rt; dn <= rt; ++dn) {
        const int fn = N + dn;
        if (fn < 0 || fn >= gf.nt1) continue;
        const T wn = dn == 0 ? T(1) : T(0.5);
        for (int dk = -rz; dk <= rz; ++dk) {
            const int fk = K + dk;
            if (fk < 0 || fk >= gf.nz1) continue;
            const T wk = dk == 0 ? T(1) : T(0.5);
            for (int dj = -rs; dj <= rs; ++dj) {
                const int fj = J + dj;
                if (fj < 0 || fj >= gf.ny1) continue;
                const T wj = dj == 0 ? T(1) : T(0.5);
                for (int di = -rs; di <= rs; ++di) {
                    const int fi = I + di;
                    if (fi < 0 || fi >= gf.nx1) continue;
                    if (!is_free<SD>(gf, fi, fj, fk, fn)) continue;
                    const T wi = di == 0 ? T(1) : T(0.5);
                    acc += wn * wk * wj * wi * rf[(((long long)fn * gf.nz1 + fk) * gf.ny1 + fj) * gf.nx1 + fi];
                }
            }
        }
    }
    return acc;
}

// (P D_c x_c) at a free fine node (i, j, k, n).
template <int SD, typename T>
__device__ __forceinline__ T prolong_node(const Geom& gf, const Geom& gc, int kind, const T* __restrict__ xc, int i,
                                          int j, int k, int n) {
    const bool cs = kind != 1, ct = kind != 0;
    int lo[4], hi[4];
    const int f[4] = {i, j, k, n};
    const bool c[4] = {cs, cs, cs && SD == 3, ct};
    for (int d = 0; d < 4; ++d) {
        if (c[d]) {
            lo[d] = f[d] >> 1;
            hi[d] = (f[d] + 1) >> 1;
        } else {
            lo[d] = hi[d] = f[d];
        }
    }
    T acc = 0;
    for (int cn = lo[3]; cn <= hi[3]; ++cn) {
        const T wn = lo[3] == hi[3] ? T(1) : T(0.5);
        for (int ck = lo[2]; ck <= hi[2]; ++ck) {
            const T wk = lo[2] == hi[2] ? T(1) : T(0.5);
            for (int cj = lo[1]; cj <= hi[1]; ++cj) {
                const T wj = lo[1] == hi[1] ? T(1) : T(0.5);
                for (int ci = lo[0]; ci <= hi[0]; ++ci) {
                    if (!is_free<SD>(gc, ci, cj, ck, cn)) continue;
                    const T wi = lo[0] == hi[0] ? T(1) : T(0.5);
                    acc += wn * wk * wj * wi * xc[(((long long)cn * gc.nz1 + ck) * gc.ny1 + cj) * gc.nx1 + ci];
                }
            }
        }
    }
    return acc;
}

// Node-parallel 27-point stencil row (plane class from n), for small levels.
template <typename T, typename LD>
__device__ __forceinline__ T row_stencil(const Geom& g, const T* __restrict__ coef, int i, int j, int n, const LD& ld) {
    const int nt = g.net;
    const long long P = (long long)g.nx1 * g.ny1;
    const long long p = (long long)j * g.nx1 + i;
    const int cls = (n == 1) ? (nt == 1 ? 3 : 0) : (n == nt ? 2 : 1);
    const T* cc = coef + (long long)cls * 27 * P + p;
    T acc = 0;
#pragma unroll
    for (int dt = 0; dt < 3; ++dt) {
        const int m = n - 1 + dt;
        if (m < 0 || m > nt) continue;
#pragma unroll
        for (int dj = 0; dj < 3; ++dj) {
            const int jj = j - 1 + dj;
            if (jj < 0 || jj >= g.ny1) continue;
#pragma unroll
            for (int di = 0; di < 3; ++di) {
                const int ii = i - 1 + di;
                if (ii < 0 || ii >= g.nx1) continue;
                acc += cc[(long long)(dt * 9 + dj * 3 + di) * P] * ld((long long)m * P + (long long)jj * g.nx1 + ii);
            }
        }
    }
    return acc;
}

// ---------------------------------------------------------------- finalisers (last block, thread 0)
template <typename T>
__device__ __forceinline__ void sm_start_finish(SmState* st_, double sum, int steps) {
    SmStateT<T>* st = smt<T>(st_);
    const T beta = (T)sqrt(sum);
    st->beta = beta;
    st->stop = !(beta > T(0) && isfinite(beta));
    if (st->rtol_rel > T(0)) {
        if (st->atol < T(0))
            st->atol = st->rtol_rel * beta;  // first start of a solve: beta = ||b||
        else if (beta <= st->atol)
            st->stop = 1;                    // converged: this and later cycles change nothing
    }
    st->s[0] = st->stop ? T(0) : T(1) / beta;
    st->kdim = steps;
    st->g[0] = beta;
    for (int q = 0; q < kMaxSmooth; ++q) st->coef[q] = T(0);
}

template <typename T>
__device__ __forceinline__ void sm_apply_finish(SmState* st_, const double* out, int j) {
    SmStateT<T>* st = smt<T>(st_);
    for (int q = 0; q <= j; ++q) st->H[q * kMaxSmooth + j] = st->s[q] * st->s[j] * (T)out[q];
}

__device__ __forceinline__ void fg_apply_finish(FgState* fs, const double* out, int j) {
    for (int q = 0; q <= j; ++q) fs->h1[q] = out[q];
}

__device__ __forceinline__ void fg_residual_finish(FgState* fs, double sum) {
    fs->beta = sqrt(sum);
    fs->res_est = fs->beta;
    fs->bad = !isfinite(fs->beta);
}

// ---------------------------------------------------------------- time-marching stencil core
// Levels whose coefficients do not change along time (extruded designs) are applied as a
// 27-point stencil: row(n, p) = sum over planes n-1, n, n+1 and the 3 x 3 neighbourhood of p.
// Coefficients are stored [class][27][P] (structure of arrays over spatial nodes p) with
// class 0: n = 1 < n_t, 1: interior, 2: n = n_t >= 2, 3: n_t == 1; prescribed rows (t = 0
// plane, spatial sink flagged in dir) are the identity.
// Asynchronous global -> shared copies of single elements (cp.async, 4 or 8 bytes); an
// invalid source copies nothing and zero-fills the destination.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc, bool valid) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int sz = valid ? (int)sizeof(T) : 0;
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async4(T* smem_dst, const T* gsrc, bool valid) {
    static_assert(sizeof(T) == 4, "4-byte elements");
    cp_async_elem<T>(smem_dst, gsrc, valid);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct MarchGrid {
    int chunk;  // planes per block
};

// Sum of c[k] v[k] over the 9 points of one plane.  FP32 pairs the terms for the packed
// two-lane FMA of sm_100+ (fma.rn.f32x2): ((c0 v0 + c2 v2 + c4 v4 + c6 v6) + (c1 v1 + ... +
// c7 v7)) + c8 v8, four instructions instead of eight; FP64 sums in order.
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pd, {%0, %1};\n\t"
        "fma.rn.f32x2 pd, pa, pb, pd;\n\t"
        "mov.b64 {%0, %1}, pd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
// The same with operands already held as register pairs: cp[i] = (c_{2i}, c_{2i+1}),
// vp[i] = (v_{2i}, v_{2i+1}) for i < 4, and the ninth term apart.
__device__ __forceinline__ float dot9p(const float2 (&cp)[4], float c8, const float2 (&vp)[4], float v8) {
    float e = 0.f, o = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) ffma2(e, o, cp[k].x, cp[k].y, vp[k].x, vp[k].y);
    return (e + o) + c8 * v8;
}

template <typename T>
__device__ __forceinline__ T dot9(const T* c, const T (&v)[9]) {
    if constexpr (std::is_same<T, float>::value) {
        float e = 0.f, o = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k += 2) ffma2(e, o, c[k], c[k + 1], v[k], v[k + 1]);
        return (e + o) + c[8] * v[8];
    } else {
        T s = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) s += c[k] * v[k];
        return s;
    }
}

// Default thread-block budget of the time-marching kernels: about two waves of 3 resident
// 256-thread blocks on each of 152 SMs, so that every block marches a long time chunk and
// its set-up (coefficients, halo cells, staging prologue) is amortised (measured on the
// 256^2 x 256 fine level: 912 blocks beat 1824 and 4096).
constexpr long long kMarchBlocks = 2 * 3 * 152;

inline __host__ MarchGrid march_grid(const Geom& g, dim3& grid, dim3& block) {
    block = dim3(32, 8, 1);
    const int gx = (g.nx1 + 31) / 32, gy = (g.ny1 + 7) / 8;
    const long long budget = g.march_blocks > 0 && g.march_blocks < kMaxBlocks ? g.march_blocks : kMarchBlocks;
    long long gz = budget / ((long long)gx * gy);
    if (gz < 1) gz = 1;
    if (gz > g.nt1) gz = g.nt1;
    const int chunk = (int)((g.nt1 + gz - 1) / gz);
    gz = (g.nt1 + chunk - 1) / chunk;
    grid = dim3(gx, gy, (unsigned)gz);
    return MarchGrid{chunk};
}

template <typename T, typename LD, typename EMIT>
__device__ __forceinline__ void march2d(const Geom& g, const T* __restrict__ coef, const unsigned char* __restrict__ dir,
                                        const LD& ld, int chunk, EMIT&& emit) {
    // A 32 x 8 tile of spatial nodes marches up the time axis over the rows [n0, n1).  Plane
    // m (tile + 1-node halo, 34 x 10 cells, at most 2 cells per thread) is staged once in
    // shared memory; each thread reads its 9-point neighbourhood of the plane and adds it to
    // the three rows it touches: the lower-plane part of row m + 1, the own-plane part of row
    // m and the upper-plane part of row m - 1, which is then complete and written.  Rows keep
    // the summation order (lower + own) + upper of a row-by-row evaluation.  Plane loads are
    // issued 3 planes ahead into a register ring; the loop is unrolled by 3 so that the ring
    // slot, the shared buffer and the three row accumulators rotate by register renaming.
    __shared__ T tile_[3][10 * 34];
    using R = typename LD::R;
    constexpr int NR = LD::NR;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int nt = g.net;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;  // planes [ms, me] feed rows [n0, n1)
    const int me = n1 <= nt ? n1 : nt;
    const long long P = (long long)g.nx1 * g.ny1;
    const bool in = i < g.nx1 && jj < g.ny1;
    const long long p = in ? (long long)jj * g.nx1 + i : 0;
    long long cell_off[2];
    bool cell_ok[2], cell_st[2];
    int cell_sm[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int cidx = tid + r * 256;
        cell_off[r] = 0;
        cell_ok[r] = false;
        cell_st[r] = cidx < 340;
        cell_sm[r] = cidx < 340 ? cidx : 0;
        if (cidx < 340) {
            const int cy = cidx / 34, cx = cidx - cy * 34;
            const int gi = i0 - 1 + cx, gj = j0 - 1 + cy;
            if (gi >= 0 && gi < g.nx1 && gj >= 0 && gj < g.ny1) {
                cell_off[r] = (long long)gj * g.nx1 + gi;
                cell_ok[r] = true;
            }
        }
    }
    const int rd = ty * 34 + tx;  // top-left of this thread's 3 x 3 neighbourhood
    T c[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) c[q] = in ? coef[(long long)(27 + q) * P + p] : T(0);
    const bool dirp = in ? (dir[p] != 0) : true;

    auto fetch = [&](int m, R (&v)[2][NR]) {
        if (m <= me) {
            const long long base = (long long)m * P;
#pragma unroll
            for (int r = 0; r < 2; ++r) ld.raw(base + cell_off[r], v[r]);
        }
    };
    // plane m: stage, refill the ring slot with plane m + 3, read the neighbourhood, add the
    // three row parts, write row m - 1 (and row n_t after the last plane)
    auto step = [&](int m, R (&slot)[2][NR], T* buf, T& a_prev, T& a_cur, T& a_next, T& c_prev, T& c_cur) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (cell_st[r]) buf[cell_sm[r]] = cell_ok[r] ? LD::combine(slot[r]) : T(0);
        fetch(m + 3, slot);
        __syncthreads();
        T v[9];
#pragma unroll
        for (int dj = 0; dj < 3; ++dj)
#pragma unroll
            for (int di = 0; di < 3; ++di) v[dj * 3 + di] = buf[rd + dj * 34 + di];
        c_cur = v[4];
        if (m >= 3 && m + 2 <= nt) {  // rows m - 1, m, m + 1 are all interior
            T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                s0 += c[k] * v[k];
                s1 += c[9 + k] * v[k];
                s2 += c[18 + k] * v[k];
            }
            a_next = s0;
            a_cur += s1;
            a_prev += s2;
        } else {
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const int r = m + 1 - part;  // row receiving this part
                T sum = 0;
                if (r >= 1 && r <= nt) {
                    const int cl = (r == 1) ? (nt == 1 ? 3 : 0) : (r == nt ? 2 : 1);
                    if (cl == 1) {
#pragma unroll
                        for (int k = 0; k < 9; ++k) sum += c[part * 9 + k] * v[k];
                    } else {
                        const T* cc = coef + (long long)(cl * 27 + part * 9) * P + p;
#pragma unroll
                        for (int k = 0; k < 9; ++k) sum += cc[(long long)k * P] * v[k];
                    }
                }
                if (part == 0)
                    a_next = sum;
                else if (part == 1)
                    a_cur += sum;
                else
                    a_prev += sum;
            }
        }
        if (in && m - 1 >= n0 && m - 1 < n1) emit((long long)(m - 1) * P + p, (m - 1 == 0 || dirp) ? c_prev : a_prev);
        if (in && m == nt && nt >= n0 && nt < n1) emit((long long)nt * P + p, dirp ? c_cur : a_cur);
    };
    R s0[2][NR], s1[2][NR], s2[2][NR];
    fetch(ms, s0);
    fetch(ms + 1, s1);
    fetch(ms + 2, s2);
    T A = 0, B = 0, Cc = 0, E0 = 0, E1 = 0, E2 = 0;
    for (int m = ms; m <= me; m += 3) {
        step(m, s0, tile_[0], A, B, Cc, E0, E1);
        if (m + 1 <= me) step(m + 1, s1, tile_[1], B, Cc, A, E1, E2);
        if (m + 2 <= me) step(m + 2, s2, tile_[2], Cc, A, B, E2, E0);
    }
}


// Smoother operator apply w = A D^-1 u on a stencil level.  The rows of interior planes read
// only interior-plane neighbours, whose Jacobi scaling is time invariant, so it is folded
// into the interior-class stencil once per design (sc[k][p] = c_k(p) d(q_k); prescribed
// spatial nodes get the identity row d(p) at the own-plane centre).  Interior rows then need
// the raw u alone, which is staged plane by plane into a ring of PF + 1 shared buffers by
// cp.async, PF planes ahead, without passing through registers.  Planes whose three rows
// are all interior and inside this block's range take a lean path (no class, range or
// boundary tests); the others use the unscaled class stencils, the scaled neighbours u d
// and the identity rows explicitly.  Rows are accumulated as in march2d.
template <typename T, int PF, typename EMIT>
__device__ __forceinline__ void march2d_scaled(const Geom& g, const T* __restrict__ sc, const T* __restrict__ coef,
                                               const unsigned char* __restrict__ dir, const T* __restrict__ u,
                                               const T* __restrict__ dinv, int chunk, EMIT&& emit) {
    constexpr int NB = PF + 3;
    static_assert((NB & (NB - 1)) == 0, "ring length must be a power of two");
    __shared__ __align__(16) T tile_[NB * 340];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int nt = g.net;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;
    const int me = n1 <= nt ? n1 : nt;
    // lean planes: rows m - 1, m, m + 1 interior and row m - 1 (written here) in range with all
    // three of its parts (planes m - 2 .. m) taken from the scaled interior stencil
    const int ml = max(n0 + 1, 5), mh = min(me, nt - 2);
    const long long P = (long long)g.nx1 * g.ny1;
    const bool in = i < g.nx1 && jj < g.ny1;
    const long long p = in ? (long long)jj * g.nx1 + i : 0;
    const T* src[2];
    bool cell_ok[2], cell_st[2];
    int cell_sm[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int cidx = tid + r * 256;
        src[r] = u;
        cell_ok[r] = false;
        cell_st[r] = cidx < 340;
        cell_sm[r] = cidx < 340 ? cidx : 0;
        if (cidx < 340) {
            const int cy = cidx / 34, cx = cidx - cy * 34;
            const int gi = i0 - 1 + cx, gj = j0 - 1 + cy;
            if (gi >= 0 && gi < g.nx1 && gj >= 0 && gj < g.ny1) {
                src[r] = u + (long long)gj * g.nx1 + gi;
                cell_ok[r] = true;
            }
        }
    }
    const int rd = ty * 34 + tx;
    T c[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) c[q] = in ? sc[(long long)q * P + p] : T(0);
    const bool dirp = in ? (dir[p] != 0) : true;
    // copies of plane m into its ring buffer; every call commits one group (possibly empty).
    // Planes are issued in order, so the cell sources advance by one plane per call.
#pragma unroll
    for (int r = 0; r < 2; ++r) src[r] += (long long)ms * P;
    auto issue = [&](int m) {
        if (m <= me) {
            T* buf = tile_ + ((m - ms) & (NB - 1)) * 340;
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (cell_st[r]) cp_async_elem<T>(buf + cell_sm[r], src[r], cell_ok[r]);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) src[r] += P;
        cp_async_commit();
    };
#pragma unroll
    for (int q = 0; q < PF; ++q) issue(ms + q);
    long long qrow = (long long)(ms - 1) * P + p;  // node index of row m - 1 at step m
    auto step = [&](int m, T& a_prev, T& a_cur, T& a_next, T& c_prev, T& c_cur) {
        cp_async_wait<PF - 1>();  // this thread's copies of plane m have landed
        __syncthreads();          // everyone's have; plane m - 1's buffer is free again
        const T* buf = tile_ + ((m - ms) & (NB - 1)) * 340;
        T v[9];
#pragma unroll
        for (int dj = 0; dj < 3; ++dj)
#pragma unroll
            for (int di = 0; di < 3; ++di) v[dj * 3 + di] = buf[rd + dj * 34 + di];
        issue(m + PF);
        c_cur = v[4];
        if (m >= ml && m <= mh) {
            a_next = dot9(c, v);
            a_cur += dot9(c + 9, v);
            a_prev += dot9(c + 18, v);
            if (in) emit(qrow, a_prev);
            qrow += P;
            return;
        }
        const bool fast = m >= 3 && m + 2 <= nt;
        if (fast) {
            T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                s0 += c[k] * v[k];
                s1 += c[9 + k] * v[k];
                s2 += c[18 + k] * v[k];
            }
            a_next = s0;
            a_cur += s1;
            a_prev += s2;
        } else {
            const T* dm = dinv + (long long)m * P;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj)
#pragma unroll
                for (int di = 0; di < 3; ++di) {
                    const int ii = i + di - 1, jn = jj + dj - 1;
                    const bool ok = in && ii >= 0 && ii < g.nx1 && jn >= 0 && jn < g.ny1;
                    v[dj * 3 + di] *= ok ? dm[(long long)jn * g.nx1 + ii] : T(0);
                }
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const int r = m + 1 - part;
                T sum = 0;
                if (r >= 1 && r <= nt) {
                    const int cl = (r == 1) ? (nt == 1 ? 3 : 0) : (r == nt ? 2 : 1);
                    const T* cc = coef + (long long)(cl * 27 + part * 9) * P + p;
#pragma unroll
                    for (int k = 0; k < 9; ++k) sum += cc[(long long)k * P] * v[k];
                }
                if (part == 0)
                    a_next = sum;
                else if (part == 1)
                    a_cur += sum;
                else
                    a_prev += sum;
            }
        }
        if (in && m - 1 >= n0 && m - 1 < n1) emit(qrow, (m - 1 == 0 || dirp) ? c_prev * dinv[qrow] : a_prev);
        if (in && m == nt && nt >= n0 && nt < n1) emit(qrow + P, dirp ? c_cur * dinv[qrow + P] : a_cur);
        qrow += P;
    };
    // three lean planes behind one wait and one barrier: the copies issued afterwards go to
    // the buffers of planes m - 3 .. m - 1 (ring of PF + 3), which every thread has finished
    // FP32: the interior stencil again as register pairs for the packed FMA
    float2 cp[3][4];
    float c8[3];
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int part = 0; part < 3; ++part) {
#pragma unroll
            for (int k = 0; k < 4; ++k) cp[part][k] = make_float2(c[part * 9 + 2 * k], c[part * 9 + 2 * k + 1]);
            c8[part] = c[part * 9 + 8];
        }
    }
    auto lean_one = [&](int m, T& a_prev, T& a_cur, T& a_next, T& c_cur) {
        const T* buf = tile_ + ((m - ms) & (NB - 1)) * 340;
        if constexpr (std::is_same<T, float>::value) {
            float2 vp[4];
            float v8;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int k0 = 2 * k, k1 = 2 * k + 1;
                vp[k].x = buf[rd + (k0 / 3) * 34 + k0 % 3];
                vp[k].y = buf[rd + (k1 / 3) * 34 + k1 % 3];
            }
            v8 = buf[rd + 2 * 34 + 2];
            c_cur = vp[2].x;  // k = 4: the centre
            a_next = dot9p(cp[0], c8[0], vp, v8);
            a_cur += dot9p(cp[1], c8[1], vp, v8);
            a_prev += dot9p(cp[2], c8[2], vp, v8);
        } else {
            T v[9];
#pragma unroll
            for (int dj = 0; dj < 3; ++dj)
#pragma unroll
                for (int di = 0; di < 3; ++di) v[dj * 3 + di] = buf[rd + dj * 34 + di];
            c_cur = v[4];
            a_next = dot9(c, v);
            a_cur += dot9(c + 9, v);
            a_prev += dot9(c + 18, v);
        }
        if (in) emit(qrow, a_prev);
        qrow += P;
    };
    T A = 0, B = 0, Cc = 0, E0 = 0, E1 = 0, E2 = 0;
    for (int m = ms; m <= me; m += 3) {
        if (m >= ml && m + 2 <= mh) {
            cp_async_wait<PF - 3>();
            __syncthreads();
            lean_one(m, A, B, Cc, E1);
            lean_one(m + 1, B, Cc, A, E2);
            lean_one(m + 2, Cc, A, B, E0);
            issue(m + PF);
            issue(m + PF + 1);
            issue(m + PF + 2);
            continue;
        }
        step(m, A, B, Cc, E0, E1);
        if (m + 1 <= me) step(m + 1, B, Cc, A, E1, E2);
        if (m + 2 <= me) step(m + 2, Cc, A, B, E2, E0);
    }
    cp_async_wait<0>();
}

}  // namespace st

namespace st {

// Givens rotation of smoother column j and, when the Arnoldi process stops (breakdown or
// the last step), the back substitution giving the final combination coefficients.
template <typename T>
__device__ inline void sm_givens_column_t(SmStateT<T>* st, int j) {
    T col[kMaxSmooth + 1];
#pragma unroll
    for (int q = 0; q <= kMaxSmooth; ++q)
        if (q <= j + 1) col[q] = st->H[q * kMaxSmooth + j];
#pragma unroll
    for (int q = 0; q < kMaxSmooth; ++q)
        if (q < j) {
            const T c = st->cs[q], s = st->sn[q];
            const T a = col[q], b = col[q + 1];
            col[q] = c * a + s * b;
            col[q + 1] = -s * a + c * b;
        }
    T a = T(0), b = T(0);
#pragma unroll
    for (int q = 0; q < kMaxSmooth; ++q)
        if (q == j) {
            a = col[q];
            b = col[q + 1];
        }
    const T r = sqrt(a * a + b * b);
    const T c = r > T(0) ? a / r : T(1), s = r > T(0) ? b / r : T(0);
    st->cs[j] = c;
    st->sn[j] = s;
    const T gj = st->g[j];
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
#pragma unroll
    for (int q = 0; q <= kMaxSmooth; ++q)
        if (q <= j + 1) st->R[q * kMaxSmooth + j] = q == j ? r : (q == j + 1 ? T(0) : col[q]);
}

template <typename T>
__device__ inline void sm_backsolve_t(SmStateT<T>* st, int k) {
    T y[kMaxSmooth];
#pragma unroll
    for (int q = kMaxSmooth - 1; q >= 0; --q) {
        y[q] = T(0);
        if (q < k) {
            T a = st->g[q];
#pragma unroll
            for (int l = 0; l < kMaxSmooth; ++l)
                if (l > q && l < k) a -= st->R[q * kMaxSmooth + l] * y[l];
            const T d = st->R[q * kMaxSmooth + q];
            y[q] = d != T(0) ? a / d : T(0);
        }
    }
#pragma unroll
    for (int q = 0; q < kMaxSmooth; ++q) st->coef[q] = q < k ? y[q] * st->s[q] : T(0);
}

template <typename T>
__device__ inline void sm_update_finish(SmState* st_, double sum, int j, int steps) {
    SmStateT<T>* st = smt<T>(st_);
    const T h = (T)sqrt(sum);
    st->H[(j + 1) * kMaxSmooth + j] = h;
    sm_givens_column_t<T>(st, j);
    const T tol = sizeof(T) == 4 ? T(1e-6) : T(1e-13);  // breakdown relative to the initial residual
    const bool conv = st->rtol_rel > T(0) && fabs(st->g[j + 1]) <= st->atol;
    const bool brk = !(h > tol * st->beta) || !isfinite(h) || conv;
    if (brk)
        st->kdim = j + 1;
    else
        st->s[j + 1] = T(1) / h;
    if (brk || j + 1 == steps) sm_backsolve_t<T>(st, j + 1);
}

__device__ inline void fg_givens_column_d(FgState* fs, int j) {
    double* H = fs->H;
    for (int q = 0; q < j; ++q) {
        const double c = fs->cs[q], s = fs->sn[q];
        const double a = H[q * kMaxRestart + j], b = H[(q + 1) * kMaxRestart + j];
        H[q * kMaxRestart + j] = c * a + s * b;
        H[(q + 1) * kMaxRestart + j] = -s * a + c * b;
    }
    const double a = H[j * kMaxRestart + j], b = H[(j + 1) * kMaxRestart + j];
    const double r = hypot(a, b);
    const double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
    fs->cs[j] = c;
    fs->sn[j] = s;
    H[j * kMaxRestart + j] = r;
    H[(j + 1) * kMaxRestart + j] = 0;
    fs->g[j + 1] = -s * fs->g[j];
    fs->g[j] = c * fs->g[j];
    fs->res_est = fabs(fs->g[j + 1]);
}

// CGS2 pass 0 done: keep the first projection in H, the second in h1.
__device__ inline void fg_pass0_finish(FgState* fs, const double* cf, const double* out, int j) {
    for (int q = 0; q <= j; ++q) {
        fs->H[q * kMaxRestart + j] = cf[q];
        fs->h1[q] = out[q];
    }
}

// CGS2 pass 1 done: complete column j, its norm and Givens rotation.
__device__ inline void fg_pass1_finish(FgState* fs, const double* cf, double sum, int j) {
    for (int q = 0; q <= j; ++q) fs->H[q * kMaxRestart + j] += cf[q];
    const double h = sqrt(sum);
    fs->H[(j + 1) * kMaxRestart + j] = h;
    fs->nrm = h;
    fg_givens_column_d(fs, j);
    fs->breakdown = !(h > 0.0);
    fs->bad = !isfinite(h) || !isfinite(fs->res_est);
}

}  // namespace st
