// Streaming Krylov kernels of the Jacobi-GMRES smoother and of the FP64 flexible GMRES
// (Sec. 3.2): basis dot products, Gram-Schmidt updates with norms, and the final linear
// combinations.  See st_stream.cuh for the access pattern.
#include <math.h>

#include "st_stream.cuh"

namespace st {

// ---------------------------------------------------------------- dots: out_q = (w, u_q), q < nq
// FIN 0: smoother column (H[q][j] = s_q s_j out_q); FIN 1: FGMRES first projection (h1).
template <typename T, int NQ, int FIN>
__global__ void __launch_bounds__(256) k_dots(long long n, const T* __restrict__ w, Ptrs<T> U, int nq, int j,
                                              void* state, RedBuf rb) {
    pdl_enter();
    if (FIN == 0) {
        const SmStateT<T>* st = smt<T>((const SmState*)state);
        if (st->stop || j >= st->kdim) return;
    }
    constexpr int W = Vec16<T>::W;
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = T(0);
    stream_loop<T>(n, [&](long long v, bool full) {
        if (full) {
            T a[W], b[NQ][W];
            Vec16<T>::get(ldv(w, v), a);
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) Vec16<T>::get(ldv(U.p[q], v), b[q]);
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) {
#pragma unroll
                    for (int l = 0; l < W; ++l) acc[q] += a[l] * b[q][l];
                }
        } else {
            for (long long e = v * W; e < n; ++e)
                for (int q = 0; q < NQ; ++q)
                    if (q < nq) acc[q] += w[e] * U.p[q][e];
        }
    });
    __shared__ double out[NQ];
    if (reduce_publish_t<T, NQ>(acc, nq, rb, out)) {
        if (threadIdx.x == 0) {
            if (FIN == 0)
                sm_apply_finish<T>((SmState*)state, out, j);
            else
                fg_apply_finish((FgState*)state, out, j);
        }
    }
}

// ---------------------------------------------------------------- update: y = a w - sum_q c_q u_q
// MODE 0: smoother step (a = s_j, c_q = H[q][j] s_q, y = u_{j+1}, norm -> Givens);
// MODE 1: FGMRES CGS2 pass 0 (y = w in place, c = h1, then dots with u_q);
// MODE 2: FGMRES CGS2 pass 1 (y = w in place, c = h1, norm, column complete).
template <typename T, int NQ, int MODE>
__global__ void __launch_bounds__(256) k_update(long long n, T* __restrict__ w, T* __restrict__ y, Ptrs<T> U, int j,
                                                int steps, void* state, RedBuf rb) {
    pdl_enter();
    constexpr int W = Vec16<T>::W;
    __shared__ T cf[NQ];
    __shared__ double cfd[NQ];
    __shared__ T a_s;
    const int nq = j + 1;
    if (MODE == 0) {
        const SmStateT<T>* st = smt<T>((const SmState*)state);
        if (st->stop || j >= st->kdim) return;
        if (threadIdx.x < nq) cf[threadIdx.x] = st->H[threadIdx.x * kMaxSmooth + j] * st->s[threadIdx.x];
        if (threadIdx.x == 0) a_s = st->s[j];
    } else {
        FgState* fs = (FgState*)state;
        if (threadIdx.x < nq) {
            cfd[threadIdx.x] = fs->h1[threadIdx.x];
            cf[threadIdx.x] = (T)fs->h1[threadIdx.x];
        }
        if (threadIdx.x == 0) a_s = T(1);
    }
    __syncthreads();
    const T a = a_s;
    constexpr int NA = MODE == 1 ? NQ : 1;
    T acc[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) acc[q] = T(0);
    stream_loop<T>(n, [&](long long v, bool full) {
        if (full) {
            T x[W], b[NQ][W];
            Vec16<T>::get(ldv_rw(w, v), x);
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) Vec16<T>::get(ldv(U.p[q], v), b[q]);
#pragma unroll
            for (int l = 0; l < W; ++l) x[l] *= a;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) {
#pragma unroll
                    for (int l = 0; l < W; ++l) x[l] -= cf[q] * b[q][l];
                }
            stv(y, v, x);
            if (MODE == 1) {
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < nq) {
#pragma unroll
                        for (int l = 0; l < W; ++l) acc[q] += x[l] * b[q][l];
                    }
            } else {
#pragma unroll
                for (int l = 0; l < W; ++l) acc[0] += x[l] * x[l];
            }
        } else {
            for (long long e = v * W; e < n; ++e) {
                T x = a * w[e];
                for (int q = 0; q < nq; ++q) x -= cf[q] * U.p[q][e];
                y[e] = x;
                if (MODE == 1) {
                    for (int q = 0; q < NQ; ++q)
                        if (q < nq) acc[q] += x * U.p[q][e];
                } else {
                    acc[0] += x * x;
                }
            }
        }
    });
    __shared__ double out[NA];
    if (reduce_publish_t<T, NA>(acc, MODE == 1 ? nq : 1, rb, out)) {
        if (threadIdx.x == 0) {
            if (MODE == 0)
                sm_update_finish<T>((SmState*)state, out[0], j, steps);
            else if (MODE == 1)
                fg_pass0_finish((FgState*)state, cfd, out, j);
            else
                fg_pass1_finish((FgState*)state, cfd, out[0], j);
        }
    }
}

// ---------------------------------------------------------------- smoother finish: x = [x +] d (.) sum_q c_q u_q
template <typename T, int NQ>
__global__ void __launch_bounds__(256) k_sm_combine(long long n, T* __restrict__ x, const T* __restrict__ dinv,
                                                    Ptrs<T> U, int zero_init, const SmState* st_) {
    pdl_enter();
    constexpr int W = Vec16<T>::W;
    const SmStateT<T>* st = smt<T>(st_);
    __shared__ T cf[NQ];
    __shared__ int kd_s;
    if (threadIdx.x == 0) kd_s = st->stop ? 0 : st->kdim;
    if (threadIdx.x < NQ) cf[threadIdx.x] = st->stop ? T(0) : st->coef[threadIdx.x];
    __syncthreads();
    const int kd = kd_s;
    stream_loop<T>(n, [&](long long v, bool full) {
        if (full) {
            T d[W], r[W], b[NQ][W];
            Vec16<T>::get(ldv(dinv, v), d);
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < kd) Vec16<T>::get(ldv(U.p[q], v), b[q]);
            if (!zero_init)
                Vec16<T>::get(ldv_rw(x, v), r);
#pragma unroll
            for (int l = 0; l < W; ++l) {
                T s = 0;
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (q < kd) s += cf[q] * b[q][l];
                r[l] = (zero_init ? T(0) : r[l]) + d[l] * s;
            }
            stv(x, v, r);
        } else {
            for (long long e = v * W; e < n; ++e) {
                T s = 0;
                for (int q = 0; q < kd; ++q) s += cf[q] * U.p[q][e];
                x[e] = (zero_init ? T(0) : x[e]) + dinv[e] * s;
            }
        }
    });
}

// ---------------------------------------------------------------- ||b||^2 -> smoother start
template <typename T>
__global__ void __launch_bounds__(256) k_sm_norm(long long n, const T* __restrict__ b, int steps, SmState* st,
                                                 RedBuf rb) {
    pdl_enter();
    constexpr int W = Vec16<T>::W;
    T acc = T(0);
    stream_loop<T>(n, [&](long long v, bool full) {
        if (full) {
            T a[W];
            Vec16<T>::get(ldv(b, v), a);
#pragma unroll
            for (int l = 0; l < W; ++l) acc += a[l] * a[l];
        } else {
            for (long long e = v * W; e < n; ++e) acc += b[e] * b[e];
        }
    });
    T d[1] = {acc};
    __shared__ double out[1];
    if (reduce_publish_t<T, 1>(d, 1, rb, out)) {
        if (threadIdx.x == 0) sm_start_finish<T>(st, out[0], steps);
    }
}

// ---------------------------------------------------------------- FGMRES x += sum_q y_q z_q
template <typename TZ, int NQ>
__global__ void __launch_bounds__(256) k_fg_combine(long long n, double* __restrict__ x, Ptrs<TZ> Z, int k,
                                                    const FgState* fs) {
    pdl_enter();
    if (k < 0) k = fs->kdone;  // graph-resident cycle: the count is read on the device (<= -k)
    __shared__ double y[NQ];
    if (threadIdx.x < NQ) y[threadIdx.x] = threadIdx.x < k ? fs->h1[threadIdx.x] : 0.0;
    __syncthreads();
    constexpr int W = 2;  // two nodes per thread (double2 for x)
    stream_loop<double>(n, [&](long long v, bool full) {
        if (full) {
            double r[W];
            Vec16<double>::get(ldv_rw(x, v), r);
            TZ b[NQ][W];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < k) {
                    b[q][0] = Z.p[q][2 * v];
                    b[q][1] = Z.p[q][2 * v + 1];
                }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < k) {
                    r[0] += y[q] * (double)b[q][0];
                    r[1] += y[q] * (double)b[q][1];
                }
            stv(x, v, r);
        } else {
            for (long long e = v * W; e < n; ++e) {
                double s = x[e];
                for (int q = 0; q < k; ++q) s += y[q] * (double)Z.p[q][e];
                x[e] = s;
            }
        }
    });
}

// ---------------------------------------------------------------- wrappers
template <typename F>
static void nq_dispatch(int nq, F&& f) {
    if (nq <= 1) f(std::integral_constant<int, 1>{});
    else if (nq <= 2) f(std::integral_constant<int, 2>{});
    else if (nq <= 4) f(std::integral_constant<int, 4>{});
    else if (nq <= 8) f(std::integral_constant<int, 8>{});
    else if (nq <= 16) f(std::integral_constant<int, 16>{});
    else f(std::integral_constant<int, 32>{});
}

template <typename T>
void launch_dots(long long n, const T* w, const Ptrs<T>& U, int nq, int j, int fin, void* state, RedBuf rb,
                 cudaStream_t s) {
    note_launch(s);
    const int blocks = stream_blocks(n, Vec16<T>::W);
    nq_dispatch(nq, [&](auto NQc) {
        constexpr int NQ = decltype(NQc)::value;
        if (fin == 0)
            launch_pdl(k_dots<T, NQ, 0>, blocks, 256, 0, s, n, w, U, nq, j, state, rb);
        else
            launch_pdl(k_dots<T, NQ, 1>, blocks, 256, 0, s, n, w, U, nq, j, state, rb);
    });
}

template <typename T>
void launch_update(long long n, T* w, T* y, const Ptrs<T>& U, int j, int steps, int mode, void* state, RedBuf rb,
                   cudaStream_t s) {
    note_launch(s);
    const int blocks = stream_blocks(n, Vec16<T>::W);
    nq_dispatch(j + 1, [&](auto NQc) {
        constexpr int NQ = decltype(NQc)::value;
        if (mode == 0)
            launch_pdl(k_update<T, NQ, 0>, blocks, 256, 0, s, n, w, y, U, j, steps, state, rb);
        else if (mode == 1)
            launch_pdl(k_update<T, NQ, 1>, blocks, 256, 0, s, n, w, y, U, j, steps, state, rb);
        else
            launch_pdl(k_update<T, NQ, 2>, blocks, 256, 0, s, n, w, y, U, j, steps, state, rb);
    });
}

template <typename T>
void launch_sm_combine(long long n, T* x, const T* dinv, const Ptrs<T>& U, int steps, bool zero_init,
                       const SmState* st, cudaStream_t s) {
    note_launch(s);
    const int blocks = stream_blocks(n, Vec16<T>::W);
    nq_dispatch(steps, [&](auto NQc) {
        constexpr int NQ = decltype(NQc)::value;
        launch_pdl(k_sm_combine<T, NQ>, blocks, 256, 0, s, n, x, dinv, U, zero_init ? 1 : 0, st);
    });
}

template <typename T>
__global__ void k_cg_begin(SmState* st, T rtol) {
    pdl_enter();
    SmStateT<T>* t = smt<T>(st);
    t->rtol_rel = rtol;
    t->atol = T(-1);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_convert(const TI* __restrict__ in, TO* __restrict__ out, long long n) {
    pdl_enter();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = (TO)in[q];
}

template <typename T>
void launch_cg_begin(SmState* st, double rtol, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_cg_begin<T>, 1, 1, 0, s, st, (T)rtol);
}

template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, long long n, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_convert<TI, TO>, stream_blocks(n, 1), 256, 0, s, in, out, n);
}

template void launch_cg_begin<double>(SmState*, double, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, long long, cudaStream_t);

template <typename T>
void launch_sm_norm(long long n, const T* b, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_sm_norm<T>, stream_blocks(n, Vec16<T>::W), 256, 0, s, n, b, steps, st, rb);
}

template <typename TZ>
void launch_fg_combine(long long n, double* x, const Ptrs<TZ>& Z, int k, const FgState* fs, cudaStream_t s) {
    note_launch(s);
    const int blocks = stream_blocks(n, 2);
    nq_dispatch(k < 0 ? -k : k, [&](auto NQc) {
        constexpr int NQ = decltype(NQc)::value;
        launch_pdl(k_fg_combine<TZ, NQ>, blocks, 256, 0, s, n, x, Z, k, fs);
    });
}

template void launch_dots<float>(long long, const float*, const Ptrs<float>&, int, int, int, void*, RedBuf, cudaStream_t);
template void launch_dots<double>(long long, const double*, const Ptrs<double>&, int, int, int, void*, RedBuf,
                                  cudaStream_t);
template void launch_update<float>(long long, float*, float*, const Ptrs<float>&, int, int, int, void*, RedBuf,
                                   cudaStream_t);
template void launch_update<double>(long long, double*, double*, const Ptrs<double>&, int, int, int, void*, RedBuf,
                                    cudaStream_t);
template void launch_sm_combine<float>(long long, float*, const float*, const Ptrs<float>&, int, bool,
                                       const SmState*, cudaStream_t);
template void launch_sm_combine<double>(long long, double*, const double*, const Ptrs<double>&, int, bool,
                                        const SmState*, cudaStream_t);
template void launch_sm_norm<float>(long long, const float*, int, SmState*, RedBuf, cudaStream_t);
template void launch_sm_norm<double>(long long, const double*, int, SmState*, RedBuf, cudaStream_t);
template void launch_fg_combine<float>(long long, double*, const Ptrs<float>&, int, const FgState*, cudaStream_t);
template void launch_fg_combine<double>(long long, double*, const Ptrs<double>&, int, const FgState*, cudaStream_t);

}  // namespace st
