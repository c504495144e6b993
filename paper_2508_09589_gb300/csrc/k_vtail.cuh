#pragma once
// Persistent coarse tail of the V-cycle (Sec. 3.2): the smoothing, residual, restriction,
// coarsest solve and prolongation of every level from `first` down to the coarsest run in
// ONE cooperative kernel, with grid-wide barriers between phases instead of separate
// launches.  These levels are small (L2 resident), so a launch per phase would cost more
// than the work.  Reductions are deterministic: every block publishes its partial sums,
// and after the barrier every block adds all partials in block order itself, so all
// blocks hold identical Hessenberg data and take identical decisions.  The smoother
// state of each level lives in shared memory.  Every barrier spin is bounded: on timeout
// the kernel sets an error flag and carries on, and the host reports ST_ERR_TIMEOUT.
#include <math.h>
#include <stddef.h>

#include <mutex>

#include "st_device.cuh"
#include "st_vtail.h"

namespace st {

struct GBar {
    unsigned* ctr;
    unsigned nb;
    unsigned epoch;
    int* err;
    unsigned long long* trace;
    int trace_cap;
    unsigned spin_limit;           // polls before a barrier wait gives up
};

__device__ __forceinline__ void gbar(GBar& b) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        b.epoch += 1;
        const unsigned target = b.epoch * b.nb;
        atomicAdd(b.ctr, 1u);
        unsigned spins = 0;
        for (;;) {
            const unsigned v = *((volatile unsigned*)b.ctr);
            if (v >= target) break;
            if (++spins > b.spin_limit) {  // default 2^24 polls, about a second: give up, report, continue
                atomicExch(b.err, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        if (b.trace && blockIdx.x == 0 && (int)b.epoch < b.trace_cap) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            b.trace[b.epoch] = t;
        }
    }
    __syncthreads();
}

// Grid sum of nq per-thread values into out[] (shared, identical in every block).
template <typename TA, int NQ>
__device__ void gsum(const TA (&v)[NQ], int nq, double* part_d, int& parity, GBar& bar, double* out) {
    __shared__ TA sm[NQ][32];
    TA* part = reinterpret_cast<TA*>(part_d);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q < nq) {
            TA a = v[q];
#pragma unroll
            for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
            if (lane == 0) sm[q][warp] = a;
        }
    }
    __syncthreads();
    TA* pb = part + (size_t)parity * kMaxBlocks * kRedQ;
    if (tid < nq) {
        TA a = 0;
        for (int w = 0; w < nw; ++w) a += sm[tid][w];
        pb[(size_t)blockIdx.x * kRedQ + tid] = a;
    }
    gbar(bar);
    const int nb = gridDim.x;
    for (int q = warp; q < nq; q += nw) out_sum_partials_t<TA>(pb, nb, q, lane, out);
    parity ^= 1;
    __syncthreads();
}

// Node coordinates from the flat index (32-bit arithmetic: the tail levels are small).
template <int SD>
__device__ __forceinline__ void decode(const Geom& g, long long q, int& i, int& j, int& k, int& n) {
    const unsigned u = (unsigned)q;
    const unsigned r1 = u / (unsigned)g.nx1;
    i = (int)(u - r1 * (unsigned)g.nx1);
    if (SD == 2) {
        const unsigned r2 = r1 / (unsigned)g.ny1;
        j = (int)(r1 - r2 * (unsigned)g.ny1);
        k = 0;
        n = (int)r2;
    } else {
        const unsigned r2 = r1 / (unsigned)g.ny1;
        j = (int)(r1 - r2 * (unsigned)g.ny1);
        const unsigned r3 = r2 / (unsigned)g.nz1;
        k = (int)(r2 - r3 * (unsigned)g.nz1);
        n = (int)r3;
    }
}

template <int SD, typename T, bool TR, typename LD>
__device__ __forceinline__ T prow(const VTail<T>& pv, const VLevel<T>& L, int i, int j, int k, int n, const LD& ld) {
    if (SD == 2 && L.dir) return row_stencil<T>(L.g, L.coef[TR ? 1 : 0], i, j, n, ld);
    if (L.lv == 0) return row_l0<SD, T, TR>(pv.op0, i, j, k, n, ld);
    OpLc<T> oc{};
    oc.g = L.g;
    oc.elem = L.elem;
    oc.tc = L.tc;
    return row_lc<SD, T, TR>(oc, i, j, k, n, ld);
}

template <typename T>
struct SmLocal {
    T H[(kMaxSmooth + 1) * kMaxSmooth];
    T s[kMaxSmooth + 1];
    T cs[kMaxSmooth], sn[kMaxSmooth], g[kMaxSmooth + 1];
    T coef[kMaxSmooth];
    T beta;
    int kdim, stop;
};

// Jacobi-GMRES smoothing on level L (zero_init: x = 0 start, u_0 = b).
template <int SD, typename T, bool TR>
__device__ void psmooth(const VTail<T>& pv, const VLevel<T>& L, bool zero_init, int steps, double* part, int& parity,
                        GBar& bar, SmLocal<T>& S) {
    const Geom& g = L.g;
    const long long N = g.nnodes;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    __shared__ double red[kMaxSmooth];
    T* U0 = zero_init ? L.b : L.U[0];
    {
        T acc = 0;
        LoadPlain<T, T> ld{L.x};
        for (long long q = t0; q < N; q += stride) {
            T r;
            if (zero_init) {
                r = L.b[q];
            } else {
                int i, j, k, n;
                decode<SD>(g, q, i, j, k, n);
                r = L.b[q] - (is_free<SD>(g, i, j, k, n) ? prow<SD, T, TR>(pv, L, i, j, k, n, ld) : L.x[q]);
                L.U[0][q] = r;
            }
            acc += r * r;
        }
        T v[1] = {acc};
        gsum<T, 1>(v, 1, part, parity, bar, red);
        if (threadIdx.x == 0) {
            const T beta = (T)sqrt(red[0]);
            S.beta = beta;
            S.stop = !(beta > T(0) && isfinite(beta));
            S.s[0] = S.stop ? T(0) : T(1) / beta;
            S.kdim = steps;
            S.g[0] = beta;
            for (int q = 0; q < kMaxSmooth; ++q) S.coef[q] = T(0);
        }
        __syncthreads();
    }
    auto U = [&](int q) -> T* { return q == 0 ? U0 : L.U[q]; };
    for (int j = 0; j < steps; ++j) {
        if (S.stop || j >= S.kdim) break;
        // w = A D^{-1} u_j and dots (w, u_q)
        {
            T acc[kMaxSmooth];
#pragma unroll
            for (int q = 0; q < kMaxSmooth; ++q) acc[q] = 0;
            LoadScaled<T> ld{U(j), L.dinv};
            for (long long q = t0; q < N; q += stride) {
                // all basis loads in flight before the stencil (one L2 round trip, not j + 1)
                T uu[kMaxSmooth];
#pragma unroll
                for (int s = 0; s < kMaxSmooth; ++s) uu[s] = s <= j ? U(s)[q] : T(0);
                int i, jj, k, n;
                decode<SD>(g, q, i, jj, k, n);
                const T w = is_free<SD>(g, i, jj, k, n) ? prow<SD, T, TR>(pv, L, i, jj, k, n, ld) : ld(q);
                L.w[q] = w;
#pragma unroll
                for (int s = 0; s < kMaxSmooth; ++s)
                    if (s <= j) acc[s] += w * uu[s];
            }
            gsum<T, kMaxSmooth>(acc, j + 1, part, parity, bar, red);
            if (threadIdx.x == 0)
                for (int s = 0; s <= j; ++s) S.H[s * kMaxSmooth + j] = S.s[s] * S.s[j] * (T)red[s];
            __syncthreads();
        }
        // u_{j+1} = s_j w - sum_q H[q][j] s_q u_q and its norm
        {
            __shared__ T cf[kMaxSmooth];
            __shared__ T sj;
            if (threadIdx.x <= j) cf[threadIdx.x] = S.H[threadIdx.x * kMaxSmooth + j] * S.s[threadIdx.x];
            if (threadIdx.x == 0) sj = S.s[j];
            __syncthreads();
            T acc = 0;
            T* un = L.U[j + 1];
            for (long long q = t0; q < N; q += stride) {
                T uu[kMaxSmooth];
#pragma unroll
                for (int s = 0; s < kMaxSmooth; ++s) uu[s] = s <= j ? U(s)[q] : T(0);
                T v = sj * L.w[q];
#pragma unroll
                for (int s = 0; s < kMaxSmooth; ++s)
                    if (s <= j) v -= cf[s] * uu[s];
                un[q] = v;
                acc += v * v;
            }
            T v[1] = {acc};
            gsum<T, 1>(v, 1, part, parity, bar, red);
            if (threadIdx.x == 0) {
                const T h = (T)sqrt(red[0]);
                S.H[(j + 1) * kMaxSmooth + j] = h;
                // Givens rotation of column j (register array, unrolled)
                T col[kMaxSmooth + 1];
#pragma unroll
                for (int q = 0; q <= kMaxSmooth; ++q) col[q] = q <= j + 1 ? S.H[q * kMaxSmooth + j] : T(0);
#pragma unroll
                for (int q = 0; q < kMaxSmooth; ++q)
                    if (q < j) {
                        const T c = S.cs[q], s = S.sn[q];
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
                S.cs[j] = c;
                S.sn[j] = s;
                const T gj = S.g[j];
                S.g[j + 1] = -s * gj;
                S.g[j] = c * gj;
#pragma unroll
                for (int q = 0; q < kMaxSmooth; ++q)
                    if (q <= j) S.H[q * kMaxSmooth + j] = q == j ? r : col[q];  // R column (upper part)
                const T tol = sizeof(T) == 4 ? T(1e-6) : T(1e-13);
                const bool brk = !(h > tol * S.beta) || !isfinite(h);
                if (brk)
                    S.kdim = j + 1;
                else
                    S.s[j + 1] = T(1) / h;
            }
            __syncthreads();
        }
    }
    // back substitution (R is stored in the upper part of H) and x update
    if (threadIdx.x == 0) {
        const int k = S.stop ? 0 : S.kdim;
        T y[kMaxSmooth];
#pragma unroll
        for (int q = kMaxSmooth - 1; q >= 0; --q) {
            y[q] = T(0);
            if (q < k) {
                T a = S.g[q];
#pragma unroll
                for (int l = 0; l < kMaxSmooth; ++l)
                    if (l > q && l < k) a -= S.H[q * kMaxSmooth + l] * y[l];
                const T d = S.H[q * kMaxSmooth + q];
                y[q] = d != T(0) ? a / d : T(0);
            }
        }
#pragma unroll
        for (int q = 0; q < kMaxSmooth; ++q) S.coef[q] = q < k ? y[q] * S.s[q] : T(0);
        S.kdim = k;
    }
    __syncthreads();
    {
        __shared__ T cf[kMaxSmooth];
        if (threadIdx.x < kMaxSmooth) cf[threadIdx.x] = S.coef[threadIdx.x];
        __syncthreads();
        const int k = S.kdim;
        for (long long q = t0; q < N; q += stride) {
            T uu[kMaxSmooth];
#pragma unroll
            for (int s = 0; s < kMaxSmooth; ++s) uu[s] = s < k ? U(s)[q] : T(0);
            const T d = L.dinv[q];
            const T x0 = zero_init ? T(0) : L.x[q];
            T v = 0;
#pragma unroll
            for (int s = 0; s < kMaxSmooth; ++s)
                if (s < k) v += cf[s] * uu[s];
            L.x[q] = x0 + d * v;
        }
    }
    gbar(bar);
}

template <int SD, typename T, bool TR>
__global__ void __launch_bounds__(256) k_vtail(const VTail<T>* __restrict__ pvp) {
    // descriptors are staged in shared memory: global copies would be reloaded after every
    // store of the node loops (the compiler cannot rule out aliasing)
    __shared__ VTail<T> pv;
    __shared__ VLevel<T> sL, sC;
    {
        const int* src = (const int*)pvp;
        int* dst = (int*)&pv;
        const int words = (int)(offsetof(VTail<T>, lv) / sizeof(int));
        for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = src[q];
    }
    auto load_level = [&](VLevel<T>& dst, int l) {
        __syncthreads();
        const int* src = (const int*)&pvp->lv[l];
        int* d = (int*)&dst;
        for (int q = threadIdx.x; q < (int)(sizeof(VLevel<T>) / sizeof(int)); q += blockDim.x) d[q] = src[q];
        __syncthreads();
    };
    __syncthreads();
    GBar bar{pv.bar, gridDim.x, 0u, pv.err, pv.trace, pv.trace_cap, pv.spin_limit};
    if (pv.trace && blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        pv.trace[0] = t;
    }
    int parity = 0;
    __shared__ SmLocal<T> S;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int Lc = pv.L - 1;
    // descend
    for (int l = pv.first; l < Lc; ++l) {
        load_level(sL, l);
        load_level(sC, l + 1);
        psmooth<SD, T, TR>(pv, sL, true, pv.steps, pv.part, parity, bar, S);
        {
            LoadPlain<T, T> ld{sL.x};
            const long long N = sL.g.nnodes;
            for (long long q = t0; q < N; q += stride) {
                int i, j, k, n;
                decode<SD>(sL.g, q, i, j, k, n);
                sL.r[q] = sL.b[q] - (is_free<SD>(sL.g, i, j, k, n) ? prow<SD, T, TR>(pv, sL, i, j, k, n, ld) : sL.x[q]);
            }
        }
        gbar(bar);
        {
            const long long N = sC.g.nnodes;
            for (long long q = t0; q < N; q += stride) {
                int i, j, k, n;
                decode<SD>(sC.g, q, i, j, k, n);
                sC.b[q] = restrict_node<SD, T>(sL.g, sC.g, sL.to_next, sL.r, i, j, k, n);
            }
        }
        gbar(bar);
    }
    // coarsest: x = Ainv b (or Ainv^T b), one warp per row
    {
        load_level(sC, Lc);
        const int n = pv.nc;
        const long long warps = stride >> 5;
        const int lane = threadIdx.x & 31;
        const double* Ainv = pv.Ainv;
        for (long long row = t0 >> 5; row < n; row += warps) {
            double a = 0;
            for (int c = lane; c < n; c += 32)
                a += (TR ? Ainv[(long long)c * n + row] : Ainv[row * (long long)n + c]) * (double)sC.b[c];
#pragma unroll
            for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
            if (lane == 0) sC.x[row] = (T)a;
        }
        gbar(bar);
    }
    // ascend
    for (int l = Lc - 1; l >= pv.first; --l) {
        load_level(sL, l);
        load_level(sC, l + 1);
        {
            const long long N = sL.g.nnodes;
            for (long long q = t0; q < N; q += stride) {
                int i, j, k, n;
                decode<SD>(sL.g, q, i, j, k, n);
                if (is_free<SD>(sL.g, i, j, k, n)) sL.x[q] += prolong_node<SD, T>(sL.g, sC.g, sL.to_next, sC.x, i, j, k, n);
            }
        }
        gbar(bar);
        psmooth<SD, T, TR>(pv, sL, false, pv.steps, pv.part, parity, bar, S);
    }
}

template <int SD, typename T, bool TR>
static int vtail_grid() {
    // blocks of one full co-resident wave (the first device that asks; computed once per
    // process, also when several server slot threads reach it together)
    static std::once_flag once;
    static int cached = 0;
    std::call_once(once, [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_vtail<SD, T, TR>, 256, 0);
        if (per < 1) per = 1;
        if (per > 2) per = 2;
        long long nb = (long long)sms * per;
        if (nb > kMaxBlocks) nb = kMaxBlocks;
        cached = (int)nb;
    });
    return cached;
}

// One (dimension, precision) pair of the launcher; the four pairs are instantiated in four
// translation units (k_vtail_2f.cu, k_vtail_2d.cu, k_vtail_3f.cu, k_vtail_3d.cu) so that the
// large tail kernels compile in parallel.
template <int SD, typename T>
int launch_vtail_sd(bool tr, const VTail<T>* dev_pv, unsigned* bar, cudaStream_t s) {
    note_launch(s);
    cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    void* args[] = {(void*)&dev_pv};
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (tr) {
        nb = vtail_grid<SD, T, true>();
        e = cudaLaunchCooperativeKernel((const void*)k_vtail<SD, T, true>, dim3(nb), dim3(256), args, 0, s);
    } else {
        nb = vtail_grid<SD, T, false>();
        e = cudaLaunchCooperativeKernel((const void*)k_vtail<SD, T, false>, dim3(nb), dim3(256), args, 0, s);
    }
    return e == cudaSuccess ? nb : -1;
}

}  // namespace st
