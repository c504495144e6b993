// Solve-phase kernels: operator applies, Jacobi diagonal, residual, multigrid
// transfers, the Jacobi-GMRES smoother, the coarsest solve and the FP64 flexible
// GMRES kernels (arXiv 2508.09589, Sec. 3.2).
#include <math.h>
#include <stdlib.h>

#include <atomic>

#include "st_device.cuh"

namespace st {

static std::atomic<long long> g_launches{0};
bool g_pdl = [] {
    const char* e = getenv("ST_PDL");
    return !(e && atoi(e) == 0);
}();
thread_local bool g_no_pdl = false;
bool g_smstep = [] {
    const char* e = getenv("ST_SMSTEP");
    return !(e && atoi(e) == 0);
}();
bool g_l0st = [] {
    const char* e = getenv("ST_L0ST");
    return !(e && atoi(e) == 0);
}();

void note_launch(cudaStream_t s, long long n) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
    g_launches += n;
}

void note_graph_launch(long long kernels) { g_launches += kernels; }

long long kernel_launches() { return g_launches.load(); }

LaunchCfg node_cfg(const Geom& g) {
    LaunchCfg c;
    c.block = dim3(32, 8, 1);
    const int gx = (g.nx1 + 31) / 32, gy = (g.ny1 + 7) / 8;
    const int planes = g.nz1 * g.nt1;
    long long gz = (long long)kMaxBlocks / ((long long)gx * gy);
    if (gz < 1) gz = 1;
    if (gz > planes) gz = planes;
    c.grid = dim3(gx, gy, (unsigned)gz);
    return c;
}

// ---------------------------------------------------------------- applies
template <int SD, typename T, int LV, bool TR>
__global__ void __launch_bounds__(256) k_apply(OpL0<T> o0, OpLc<T> oc, const T* __restrict__ x, T* __restrict__ y) {
    pdl_enter();
    const Geom& g = LV == 0 ? o0.g : oc.g;
    LoadPlain<T, T> ld{x};
    ST_NODE_LOOP_BEGIN(g)
    T v;
    if (is_free<SD>(g, i_, j_, k_, n_))
        v = op_row<SD, T, LV, TR>(o0, oc, i_, j_, k_, n_, ld);
    else
        v = x[idx_];
    y[idx_] = v;
    ST_NODE_LOOP_END
}

template <int SD, typename T, int LV>
__global__ void __launch_bounds__(256) k_diag(OpL0<T> o0, OpLc<T> oc, T* __restrict__ d, int invert) {
    pdl_enter();
    const Geom& g = LV == 0 ? o0.g : oc.g;
    ST_NODE_LOOP_BEGIN(g)
    T v = T(1);
    if (is_free<SD>(g, i_, j_, k_, n_)) {
        if constexpr (LV == 0)
            v = diag_l0<SD, T>(o0, i_, j_, k_, n_);
        else
            v = diag_lc<SD, T>(oc, i_, j_, k_, n_);
    }
    d[idx_] = invert ? T(1) / v : v;
    ST_NODE_LOOP_END
}

template <int SD, typename T, int LV, bool TR>
__global__ void __launch_bounds__(256) k_residual(OpL0<T> o0, OpLc<T> oc, const T* __restrict__ b,
                                                  const T* __restrict__ x, T* __restrict__ r) {
    pdl_enter();
    const Geom& g = LV == 0 ? o0.g : oc.g;
    LoadPlain<T, T> ld{x};
    ST_NODE_LOOP_BEGIN(g)
    T v;
    if (is_free<SD>(g, i_, j_, k_, n_))
        v = b[idx_] - op_row<SD, T, LV, TR>(o0, oc, i_, j_, k_, n_, ld);
    else
        v = b[idx_] - x[idx_];
    r[idx_] = v;
    ST_NODE_LOOP_END
}

// ---------------------------------------------------------------- transfers
// kind: 0 = space (all spatial axes halved), 1 = time, 2 = both.
// Restriction r_c = D_c P^T D_f r_f (P trilinear, vertex nested).
template <int SD, typename T>
__global__ void __launch_bounds__(256) k_restrict(Geom gf, Geom gc, int kind, const T* __restrict__ rf,
                                                  T* __restrict__ rc) {
    pdl_enter();
    ST_NODE_LOOP_BEGIN(gc)
    rc[idx_] = restrict_node<SD, T>(gf, gc, kind, rf, i_, j_, k_, n_);
    ST_NODE_LOOP_END
}

// Prolongation x_f += D_f P D_c x_c.
template <int SD, typename T>
__global__ void __launch_bounds__(256) k_prolong(Geom gf, Geom gc, int kind, const T* __restrict__ xc,
                                                 T* __restrict__ xf) {
    pdl_enter();
    ST_NODE_LOOP_BEGIN(gf)
    if (is_free<SD>(gf, i_, j_, k_, n_)) xf[idx_] += prolong_node<SD, T>(gf, gc, kind, xc, i_, j_, k_, n_);
    ST_NODE_LOOP_END
}

// ---------------------------------------------------------------- Jacobi-GMRES smoother
// Right-preconditioned GMRES on A D^{-1} y = b - A x0, x = x0 + D^{-1} y, with the
// basis kept unnormalised (u_j) and scales s_j = 1 / ||u_j|| (classical Gram-Schmidt,
// one reduction per step); Givens rotations are applied as columns arrive.
template <int SD, typename T, int LV, bool TR, bool ZERO>
__global__ void __launch_bounds__(256) k_sm_start(OpL0<T> o0, OpLc<T> oc, const T* __restrict__ b,
                                                  const T* __restrict__ x, T* __restrict__ u0, int steps,
                                                  SmState* st, RedBuf rb) {
    pdl_enter();
    const Geom& g = LV == 0 ? o0.g : oc.g;
    LoadPlain<T, T> ld{x};
    double acc[1] = {0.0};
    T accT = T(0);
    ST_NODE_LOOP_BEGIN(g)
    T r;
    if (ZERO) {
        r = b[idx_];
    } else {
        if (is_free<SD>(g, i_, j_, k_, n_))
            r = b[idx_] - op_row<SD, T, LV, TR>(o0, oc, i_, j_, k_, n_, ld);
        else
            r = b[idx_] - x[idx_];
        u0[idx_] = r;
    }
    accT += r * r;
    ST_NODE_LOOP_END
    T accv[1] = {accT};
    (void)acc;
    __shared__ double out[1];
    if (reduce_publish_t<T, 1>(accv, 1, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sm_start_finish<T>(st, out[0], steps);
    }
}

// ---------------------------------------------------------------- coarsest solve
template <typename T>
__global__ void k_coarse_gemv(const double* __restrict__ Ainv, int n, const T* __restrict__ b, T* __restrict__ x) {
    pdl_enter();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double* row = Ainv + (long long)warp * n;
    double a = 0;
    for (int c = lane; c < n; c += 32) a += row[c] * (double)b[c];
#pragma unroll
    for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) x[warp] = (T)a;
}

template <typename T>
__global__ void k_coarse_gemv_t(const double* __restrict__ Ainv, int n, const T* __restrict__ b, T* __restrict__ x) {
    pdl_enter();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double a = 0;
    for (int c = 0; c < n; ++c) a += Ainv[(long long)c * n + r] * (double)b[c];
    x[r] = (T)a;
}

// ---------------------------------------------------------------- FGMRES (FP64)
struct VPtrs {
    double* v[kMaxRestart + 1];
};

template <typename TZ>
struct ZPtrs {
    TZ* z[kMaxRestart];
};

__device__ void fg_givens_column(FgState* fs, int j) {
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

static_assert(kRedQ >= kMaxRestart && kRedQ >= kMaxSmooth, "partial-sum stride too small");

template <typename TZ>
__global__ void __launch_bounds__(256) k_fg_normalize(Geom g, const double* __restrict__ w,
                                                      double* __restrict__ vn, TZ* __restrict__ bmg,
                                                      const FgState* fs) {
    pdl_enter();
    const double h = fs->nrm;
    const double inv = h > 0 ? 1.0 / h : 0.0;
    ST_NODE_LOOP_BEGIN(g)
    const double v = w[idx_] * inv;
    vn[idx_] = v;
    bmg[idx_] = (TZ)v;
    ST_NODE_LOOP_END
}

__global__ void k_fg_backsolve(FgState* fs, int k) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (k < 0) k = fs->kdone;  // graph-resident cycle: the iterations it completed
    for (int q = k - 1; q >= 0; --q) {
        double a = fs->g[q];
        for (int l = q + 1; l < k; ++l) a -= fs->H[q * kMaxRestart + l] * fs->h1[l];
        const double d = fs->H[q * kMaxRestart + q];
        fs->h1[q] = d != 0 ? a / d : 0.0;  // y stored in h1
    }
}

// ---------------------------------------------------------------- graph-resident cycle control
__global__ void k_fg_begin(FgState* fs, double tol, int max_it, cudaGraphConditionalHandle hw) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double beta = fs->beta;
    const bool go = beta == beta && !fs->bad && beta > tol && fs->its < max_it;
    fs->kdone = 0;
    fs->cont = go ? 1 : 0;
    cudaGraphSetConditional(hw, go ? 1u : 0u);
}

__global__ void k_fg_setj(const FgState* fs, cudaGraphConditionalHandle hs) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(hs, (unsigned)fs->kdone);
}

__global__ void k_fg_check(FgState* fs, int j, double tol, int max_it, int m) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fs->its += 1;
    fs->kdone = j + 1;
    const bool stop = fs->bad || fs->res_est <= tol || fs->breakdown || fs->its >= max_it || j + 1 >= m;
    fs->cont = stop ? 0 : 1;
}

__global__ void k_fg_loop(const FgState* fs, cudaGraphConditionalHandle hw) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(hw, fs->cont ? 1u : 0u);
}

void launch_fg_begin(FgState* fs, double tol, int max_it, cudaGraphConditionalHandle hw, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_fg_begin, 1, 32, 0, s, fs, tol, max_it, hw);
}
void launch_fg_setj(const FgState* fs, cudaGraphConditionalHandle hs, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_fg_setj, 1, 32, 0, s, fs, hs);
}
void launch_fg_check(FgState* fs, int j, double tol, int max_it, int m, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_fg_check, 1, 32, 0, s, fs, j, tol, max_it, m);
}
void launch_fg_loop(const FgState* fs, cudaGraphConditionalHandle hw, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_fg_loop, 1, 32, 0, s, fs, hw);
}

template <int SD, bool TR>
__global__ void __launch_bounds__(256) k_fg_residual(OpL0<double> op, const double* __restrict__ f,
                                                     const double* __restrict__ x, double* __restrict__ r,
                                                     FgState* fs, RedBuf rb) {
    pdl_enter();
    const Geom& g = op.g;
    LoadPlain<double, double> ld{x};
    double acc[1] = {0.0};
    ST_NODE_LOOP_BEGIN(g)
    double v;
    if (is_free<SD>(g, i_, j_, k_, n_))
        v = f[idx_] - row_l0<SD, double, TR>(op, i_, j_, k_, n_, ld);
    else
        v = f[idx_] - x[idx_];
    r[idx_] = v;
    acc[0] += v * v;
    ST_NODE_LOOP_END
    __shared__ double out[1];
    if (reduce_publish<1>(acc, 1, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) fg_residual_finish(fs, out[0]);
    }
}

template <typename TZ>
__global__ void __launch_bounds__(256) k_fg_start(Geom g, double* __restrict__ v0, TZ* __restrict__ bmg,
                                                  FgState* fs) {
    pdl_enter();
    const double beta = fs->beta;
    const double inv = beta > 0 ? 1.0 / beta : 0.0;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        // g is read by later kernels only
        fs->g[0] = beta;
        for (int q = 1; q <= kMaxRestart; ++q) fs->g[q] = 0.0;
        fs->breakdown = 0;
    }
    ST_NODE_LOOP_BEGIN(g)
    const double v = v0[idx_] * inv;
    v0[idx_] = v;
    bmg[idx_] = (TZ)v;
    ST_NODE_LOOP_END
}

__global__ void __launch_bounds__(256) k_dot64(Geom g, const double* __restrict__ a, const double* __restrict__ b,
                                               double* out_d, RedBuf rb) {
    pdl_enter();
    double acc[1] = {0.0};
    ST_NODE_LOOP_BEGIN(g)
    acc[0] += a[idx_] * b[idx_];
    ST_NODE_LOOP_END
    __shared__ double out[1];
    if (reduce_publish<1>(acc, 1, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) *out_d = out[0];
    }
}

template <int SD>
__global__ void __launch_bounds__(256) k_mask_copy(Geom g, const double* __restrict__ src, double* __restrict__ dst) {
    pdl_enter();
    ST_NODE_LOOP_BEGIN(g)
    dst[idx_] = is_free<SD>(g, i_, j_, k_, n_) ? src[idx_] : 0.0;
    ST_NODE_LOOP_END
}


// ---------------------------------------------------------------- time-marching variants
// Used when the level carries 27-point stencils (extruded design, 2 spatial dimensions).
template <typename T>
__global__ void __launch_bounds__(256) km_apply(Geom g, const T* __restrict__ coef, const unsigned char* __restrict__ dir,
                                                int chunk, const T* __restrict__ x, T* __restrict__ y) {
    pdl_enter();
    LoadPlain<T, T> ld{x};
    march2d<T>(g, coef, dir, ld, chunk, [&](long long q, T v) { y[q] = v; });
}

template <typename T>
__global__ void __launch_bounds__(256) km_residual(Geom g, const T* __restrict__ coef,
                                                   const unsigned char* __restrict__ dir, int chunk,
                                                   const T* __restrict__ b, const T* __restrict__ x,
                                                   T* __restrict__ r) {
    pdl_enter();
    LoadPlain<T, T> ld{x};
    march2d<T>(g, coef, dir, ld, chunk, [&](long long q, T v) { r[q] = b[q] - v; });
}

template <typename T>
__global__ void __launch_bounds__(256) km_sm_start(Geom g, const T* __restrict__ coef,
                                                   const unsigned char* __restrict__ dir, int chunk,
                                                   const T* __restrict__ b, const T* __restrict__ x,
                                                   T* __restrict__ u0, int steps, SmState* st, RedBuf rb) {
    pdl_enter();
    LoadPlain<T, T> ld{x};
    T accT = T(0);
    march2d<T>(g, coef, dir, ld, chunk, [&](long long q, T v) {
        const T r = b[q] - v;
        u0[q] = r;
        accT += r * r;
    });
    T acc[1] = {accT};
    __shared__ double out[1];
    if (reduce_publish_t<T, 1>(acc, 1, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sm_start_finish<T>(st, out[0], steps);
    }
}

__global__ void __launch_bounds__(256) km_fg_residual(Geom g, const double* __restrict__ coef,
                                                      const unsigned char* __restrict__ dir, int chunk,
                                                      const double* __restrict__ f, const double* __restrict__ x,
                                                      double* __restrict__ r, FgState* fs, RedBuf rb) {
    pdl_enter();
    LoadPlain<double, double> ld{x};
    double acc[1] = {0.0};
    march2d<double>(g, coef, dir, ld, chunk, [&](long long q, double v) {
        const double rr = f[q] - v;
        r[q] = rr;
        acc[0] += rr * rr;
    });
    __shared__ double out[1];
    if (reduce_publish<1>(acc, 1, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) fg_residual_finish(fs, out[0]);
    }
}


// Smoother step apply only (dots in a streaming kernel): w = A (D^{-1} u_j).
template <typename T>
__global__ void __launch_bounds__(256) km_sm_applyw(Geom g, const T* __restrict__ coef,
                                                    const unsigned char* __restrict__ dir, int chunk,
                                                    const T* __restrict__ dinv, const T* __restrict__ uj,
                                                    T* __restrict__ w, int j, const SmState* st) {
    pdl_enter();
    if (smt<T>(st)->stop || j >= smt<T>(st)->kdim) return;
    LoadScaled<T> ld{uj, dinv};
    march2d<T>(g, coef, dir, ld, chunk, [&](long long q, T v) { w[q] = v; });
}

// The same with the interior Jacobi scaling folded into the stencil (reads u_j only).
template <typename T>
__global__ void __launch_bounds__(256) km_sm_applyw_sc(Geom g, const T* __restrict__ sc, const T* __restrict__ coef,
                                                       const unsigned char* __restrict__ dir, int chunk,
                                                       const T* __restrict__ dinv, const T* __restrict__ uj,
                                                       T* __restrict__ w, int j, const SmState* st) {
    pdl_enter();
    if (smt<T>(st)->stop || j >= smt<T>(st)->kdim) return;
    constexpr int PF = sizeof(T) == 4 ? 13 : 5;  // planes in flight per block (ring of PF + 3)
    march2d_scaled<T, PF>(g, sc, coef, dir, uj, dinv, chunk, [&](long long q, T v) { w[q] = v; });
}

template <int SD, typename T, int LV, bool TR>
__global__ void __launch_bounds__(256) k_sm_applyw(OpL0<T> o0, OpLc<T> oc, const T* __restrict__ dinv,
                                                   const T* __restrict__ uj, T* __restrict__ w, int j,
                                                   const SmState* st) {
    pdl_enter();
    if (smt<T>(st)->stop || j >= smt<T>(st)->kdim) return;
    const Geom& g = LV == 0 ? o0.g : oc.g;
    LoadScaled<T> ld{uj, dinv};
    ST_NODE_LOOP_BEGIN(g)
    w[idx_] = is_free<SD>(g, i_, j_, k_, n_) ? op_row<SD, T, LV, TR>(o0, oc, i_, j_, k_, n_, ld) : ld(idx_);
    ST_NODE_LOOP_END
}

// FGMRES: w = A z (FP64) and the copy of z into the basis Z_j.
template <typename TZ>
__global__ void __launch_bounds__(256) km_fg_apply(Geom g, const double* __restrict__ coef,
                                                   const unsigned char* __restrict__ dir, int chunk,
                                                   const TZ* __restrict__ z, TZ* __restrict__ zstore,
                                                   double* __restrict__ w) {
    pdl_enter();
    LoadPlain<double, TZ> ld{z};
    march2d<double>(g, coef, dir, ld, chunk, [&](long long q, double v) {
        w[q] = v;
        zstore[q] = z[q];
    });
}

template <int SD, typename TZ, bool TR>
__global__ void __launch_bounds__(256) k_fg_apply(OpL0<double> op, const TZ* __restrict__ z, TZ* __restrict__ zstore,
                                                  double* __restrict__ w) {
    pdl_enter();
    const Geom& g = op.g;
    LoadPlain<double, TZ> ld{z};
    ST_NODE_LOOP_BEGIN(g)
    w[idx_] = is_free<SD>(g, i_, j_, k_, n_) ? row_l0<SD, double, TR>(op, i_, j_, k_, n_, ld) : (double)z[idx_];
    zstore[idx_] = z[idx_];
    ST_NODE_LOOP_END
}

// ---------------------------------------------------------------- launch wrappers
#define ST_SD_DISPATCH(sd, ...) \
    do {                        \
        if ((sd) == 2) {        \
            constexpr int SD = 2; \
            __VA_ARGS__;        \
        } else {                \
            constexpr int SD = 3; \
            __VA_ARGS__;        \
        }                       \
    } while (0)

template <typename T>
static OpLc<T> dummy_lc(const Geom& g) {
    OpLc<T> o{};
    o.g = g;
    return o;
}
template <typename T>
static OpL0<T> dummy_l0(const Geom& g) {
    OpL0<T> o{};
    o.g = g;
    return o;
}

template <typename T>
void launch_apply_l0(int sd, const OpL0<T>& op, bool tr, const T* x, T* y, cudaStream_t s) {
    note_launch(s);
    if (sd == 2 && op.st_dir) {
        dim3 grid, block;
        const MarchGrid mg = march_grid(op.g, grid, block);
        launch_pdl(km_apply<T>, grid, block, 0, s, op.g, op.st_coef[tr ? 1 : 0], op.st_dir, mg.chunk, x, y);
        return;
    }
    if constexpr (std::is_same<T, double>::value) {
        const void* vecs[2] = {x, y};
        if (fg_march_usable(sd, op, vecs, 2)) {
            launch_fg_march<double>(sd, 0, tr, op, x, nullptr, nullptr, y, nullptr, RedBuf{}, s);
            return;
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        const void* vecs[2] = {x, y};
        if (l0_march_usable(sd, op, vecs, 2)) {
            if (sd == 2)
                launch_l0st(3, tr, op, x, nullptr, nullptr, y, 0, 0, nullptr, RedBuf{}, s);
            else
                launch_l0x3(3, tr, op, x, nullptr, nullptr, y, 0, 0, nullptr, RedBuf{}, s);
            return;
        }
    }
    const LaunchCfg c = node_cfg(op.g);
    const OpLc<T> oc = dummy_lc<T>(op.g);
    ST_SD_DISPATCH(sd, if (tr) launch_pdl(k_apply<SD, T, 0, true>, c.grid, c.block, 0, s, op, oc, x, y);
                   else launch_pdl(k_apply<SD, T, 0, false>, c.grid, c.block, 0, s, op, oc, x, y));
}
template <typename T>
void launch_apply_lc(int sd, const OpLc<T>& op, bool tr, const T* x, T* y, cudaStream_t s) {
    note_launch(s);
    if (sd == 2 && op.st_dir) {
        dim3 grid, block;
        const MarchGrid mg = march_grid(op.g, grid, block);
        launch_pdl(km_apply<T>, grid, block, 0, s, op.g, op.st_coef[tr ? 1 : 0], op.st_dir, mg.chunk, x, y);
        return;
    }
    if constexpr (std::is_same<T, float>::value) {
        const void* vecs[2] = {x, y};
        if (sd == 3 && g_l0st && lcx3_usable(op, vecs, 2)) {
            launch_lcx3(3, tr, op, x, nullptr, nullptr, y, 0, 0, nullptr, RedBuf{}, s);
            return;
        }
        if (sd == 2 && g_l0st && lcst_usable(op, vecs, 2)) {
            launch_lcst(3, tr, op, x, nullptr, nullptr, y, 0, 0, nullptr, RedBuf{}, s);
            return;
        }
    }
    const LaunchCfg c = node_cfg(op.g);
    const OpL0<T> o0 = dummy_l0<T>(op.g);
    ST_SD_DISPATCH(sd, if (tr) launch_pdl(k_apply<SD, T, 1, true>, c.grid, c.block, 0, s, o0, op, x, y);
                   else launch_pdl(k_apply<SD, T, 1, false>, c.grid, c.block, 0, s, o0, op, x, y));
}
template <typename T>
void launch_diag_l0(int sd, const OpL0<T>& op, T* d, bool invert, cudaStream_t s) {
    if (sd == 2 && op.st_dir) {
        launch_stencil_diag<T>(op.g, op.st_coef[0], op.st_dir, d, invert, s);
        return;
    }
    note_launch(s);
    const LaunchCfg c = node_cfg(op.g);
    const OpLc<T> oc = dummy_lc<T>(op.g);
    ST_SD_DISPATCH(sd, launch_pdl(k_diag<SD, T, 0>, c.grid, c.block, 0, s, op, oc, d, invert ? 1 : 0));
}
template <typename T>
void launch_diag_lc(int sd, const OpLc<T>& op, T* d, bool invert, cudaStream_t s) {
    if (sd == 2 && op.st_dir) {
        launch_stencil_diag<T>(op.g, op.st_coef[0], op.st_dir, d, invert, s);
        return;
    }
    note_launch(s);
    const LaunchCfg c = node_cfg(op.g);
    const OpL0<T> o0 = dummy_l0<T>(op.g);
    ST_SD_DISPATCH(sd, launch_pdl(k_diag<SD, T, 1>, c.grid, c.block, 0, s, o0, op, d, invert ? 1 : 0));
}
template <typename T>
void launch_residual(int sd, int lvl, const OpL0<T>& o0, const OpLc<T>& oc, bool tr, const T* b, const T* x, T* r,
                     cudaStream_t s) {
    note_launch(s);
    {
        const Geom& g = lvl == 0 ? o0.g : oc.g;
        const unsigned char* dir = lvl == 0 ? o0.st_dir : oc.st_dir;
        if (sd == 2 && dir) {
            const T* coef = lvl == 0 ? o0.st_coef[tr ? 1 : 0] : oc.st_coef[tr ? 1 : 0];
            dim3 grid, block;
            const MarchGrid mg = march_grid(g, grid, block);
            launch_pdl(km_residual<T>, grid, block, 0, s, g, coef, dir, mg.chunk, b, x, r);
            return;
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        const void* vecs[3] = {b, x, r};
        if (lvl == 0 && l0_march_usable(sd, o0, vecs, 3)) {
            if (sd == 2)
                launch_l0st(1, tr, o0, x, nullptr, b, r, 0, 0, nullptr, RedBuf{}, s);
            else
                launch_l0x3(1, tr, o0, x, nullptr, b, r, 0, 0, nullptr, RedBuf{}, s);
            return;
        }
        if (lvl > 0 && sd == 3 && g_l0st && lcx3_usable(oc, vecs, 3)) {
            launch_lcx3(1, tr, oc, x, nullptr, b, r, 0, 0, nullptr, RedBuf{}, s);
            return;
        }
        if (lvl > 0 && sd == 2 && !oc.st_dir && g_l0st && lcst_usable(oc, vecs, 3)) {
            launch_lcst(1, tr, oc, x, nullptr, b, r, 0, 0, nullptr, RedBuf{}, s);
            return;
        }
    }
    const LaunchCfg c = node_cfg(lvl == 0 ? o0.g : oc.g);
    if (lvl == 0) {
        ST_SD_DISPATCH(sd, if (tr) launch_pdl(k_residual<SD, T, 0, true>, c.grid, c.block, 0, s, o0, oc, b, x, r);
                       else launch_pdl(k_residual<SD, T, 0, false>, c.grid, c.block, 0, s, o0, oc, b, x, r));
    } else {
        ST_SD_DISPATCH(sd, if (tr) launch_pdl(k_residual<SD, T, 1, true>, c.grid, c.block, 0, s, o0, oc, b, x, r);
                       else launch_pdl(k_residual<SD, T, 1, false>, c.grid, c.block, 0, s, o0, oc, b, x, r));
    }
}
template <typename T>
void launch_restrict(const Geom& gf, const Geom& gc, int kind, int sd, const T* rf, T* rc, cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(gc);
    ST_SD_DISPATCH(sd, launch_pdl(k_restrict<SD, T>, c.grid, c.block, 0, s, gf, gc, kind, rf, rc));
}
template <typename T>
void launch_prolong(const Geom& gf, const Geom& gc, int kind, int sd, const T* xc, T* xf, cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(gf);
    ST_SD_DISPATCH(sd, launch_pdl(k_prolong<SD, T>, c.grid, c.block, 0, s, gf, gc, kind, xc, xf));
}

// Timing event on stream s: an event node when the stream is being captured into a graph,
// a plain record otherwise.  A failure only loses the sample (the reader skips pairs whose
// elapsed time cannot be read), so its error is cleared here.
static void record_timing_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (cudaEventRecordWithFlags(e, s, flags) != cudaSuccess) cudaGetLastError();
}

// The level-0 space-time kernels (k_l0st.cu) where the instantiation can use them (FP32,
// 2-D, level 0) and on is set; false when the caller must launch the node-parallel kernel.
template <int SD, typename T, int LV>
static bool launch_l0st_if(bool on, int mode, bool tr, const OpL0<T>& o0, const OpLc<T>& oc, const T* u,
                           const T* dinv, const T* b, T* out, int j, int steps, SmState* st, RedBuf rb,
                           cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (on) {
            if constexpr (LV == 0 && SD == 2)
                launch_l0st(mode, tr, o0, u, dinv, b, out, j, steps, st, rb, s);
            else if constexpr (LV == 0)
                launch_l0x3(mode, tr, o0, u, dinv, b, out, j, steps, st, rb, s);
            else if constexpr (SD == 3)
                launch_lcx3(mode, tr, oc, u, dinv, b, out, j, steps, st, rb, s);
            else
                launch_lcst(mode, tr, oc, u, dinv, b, out, j, steps, st, rb, s);
            return true;
        }
    }
    return false;
}

// Whether the level-0 marching kernels of k_l0st.cu (space-time 2-D designs) or k_l0x3.cu
// (extruded 3-D designs) take these vectors.
static bool l0_march_usable(int sd, const OpL0<float>& op, const void* const* vecs, int nvec) {
    if (!g_l0st) return false;
    return sd == 2 ? l0st_usable(op, vecs, nvec) : l0x3_usable(op, vecs, nvec);
}

template <int SD, typename T, int LV, bool TR>
static void smooth_impl(const OpL0<T>& o0, const OpLc<T>& oc, const T* b, T* x, const T* dinv, Basis<T> U, T* w,
                        T* w2, int steps, bool zero_init, SmState* st, RedBuf rb, cudaStream_t s,
                        cudaEvent_t* ev, const T* sc) {
    const Geom& g = LV == 0 ? o0.g : oc.g;
    const long long N = g.nnodes;
    const LaunchCfg c = node_cfg(g);
    const unsigned char* dir = LV == 0 ? o0.st_dir : oc.st_dir;
    const bool march = SD == 2 && dir != nullptr;
    const T* coef = march ? (LV == 0 ? o0.st_coef[TR ? 1 : 0] : oc.st_coef[TR ? 1 : 0]) : nullptr;
    dim3 mgrid, mblock;
    const MarchGrid mg = march_grid(g, mgrid, mblock);
    if (zero_init) U.u[0] = const_cast<T*>(b);
    Ptrs<T> P{};
    for (int q = 0; q <= steps; ++q) P.p[q] = U.u[q];
    // FP32 levels of a space-time 2-D design (level 0) or an extruded 3-D design (every level
    // with extracted stencils): the time-marching kernels of k_l0st.cu and k_l0x3.cu
    bool l0st = false;
    if constexpr (std::is_same<T, float>::value) {
        const void* vecs[4 + kMaxSmooth + 1] = {b, x, dinv, w};
        for (int q = 0; q <= steps; ++q) vecs[4 + q] = U.u[q];
        if constexpr (LV == 0)
            l0st = !march && l0_march_usable(SD, o0, vecs, 4 + steps + 1);
        else
            l0st = g_l0st && !march &&
                   (SD == 3 ? lcx3_usable(oc, vecs, 4 + steps + 1) : lcst_usable(oc, vecs, 4 + steps + 1));
    }
    // The fused Arnoldi step (one pass per step, halo recomputed) only pays on tiny, latency
    // bound levels; on large levels the split apply / dots / update kernels stream faster.
    constexpr long long kFusedMaxNodes = 15000;
    const bool fused = march && std::is_same<T, float>::value && w2 != nullptr && steps >= 2 && steps + 1 <= 16 &&
                       N <= kFusedMaxNodes && ev == nullptr;
    if (zero_init) {
        launch_sm_norm<T>(N, b, steps, st, rb, s);
    } else {
        note_launch(s);
        if (march)
            launch_pdl(km_sm_start<T>, mgrid, mblock, 0, s, g, coef, dir, mg.chunk, b, x, U.u[0], steps, st, rb);
        else if (!launch_l0st_if<SD, T, LV>(l0st, 2, TR, o0, oc, x, nullptr, b, U.u[0], 0, steps, st, rb, s))
            launch_pdl(k_sm_start<SD, T, LV, TR, false>, c.grid, c.block, 0, s, o0, oc, b, x, U.u[0], steps, st, rb);
    }
    if (fused) {
        if constexpr (std::is_same<T, float>::value) {
            // step 0: w = A D^{-1} u_0 and (w, u_0); then fused steps j -> j+1; the last
            // update only closes the Hessenberg matrix (norm of u_m) before the combination.
            note_launch(s);
            launch_pdl(km_sm_applyw<T>, mgrid, mblock, 0, s, g, coef, dir, mg.chunk, dinv, U.u[0], w, 0, st);
            launch_dots<T>(N, w, P, 1, 0, 0, st, rb, s);
            T* wc = w;
            T* wn = w2;
            for (int j = 0; j + 1 < steps; ++j) {
                launch_arnoldi(g, coef, dir, dinv, P, wc, wn, j, st, rb, s);
                T* t = wc;
                wc = wn;
                wn = t;
            }
            launch_update<T>(N, wc, U.u[steps], P, steps - 1, steps, 0, st, rb, s);
            launch_sm_combine<T>(N, x, dinv, P, steps, zero_init, st, s);
            return;
        }
    }
    // FP32 only: in FP64 the ring of up to 11 staged vectors leaves one block per SM, and the
    // separate kernels below are faster (measured 1.79 s against 2.18 s per c1 step)
    if constexpr (std::is_same<T, float>::value) {
        if (march && sc && w2 != nullptr && g_smstep && sm_step_aligned<T>(P, steps, w, w2, N, g.plane)) {
            // one kernel per Arnoldi step (update of step j - 1, apply and dots of step j), w_j
            // alternating between w and w2; then the last update (norm of u_steps and the back
            // substitution) and the combination
            const T* sco = sc + (TR ? 27 * g.plane : 0);
            T* wb[2] = {w, w2};
            for (int j = 0; j < steps; ++j) {
                if (ev) record_timing_event(ev[2 * j], s);
                launch_sm_step<T>(g, sco, coef, dir, dinv, P, j ? wb[(j - 1) & 1] : nullptr, wb[j & 1], j, steps,
                                  st, rb, s);
                if (ev) record_timing_event(ev[2 * j + 1], s);
            }
            launch_update<T>(N, wb[(steps - 1) & 1], U.u[steps], P, steps - 1, steps, 0, st, rb, s);
            launch_sm_combine<T>(N, x, dinv, P, steps, zero_init, st, s);
            return;
        }
    }
    // Arnoldi step j: w = A D^-1 u_j (stencil kernel), the dots (w, u_q), then the update
    // u_{j+1} = w - sum h_q u_q with its norm, each a separate bandwidth-efficient kernel
    for (int j = 0; j < steps; ++j) {
        note_launch(s);
        // optional timing events around the operator apply (event nodes when captured)
        if (ev) record_timing_event(ev[2 * j], s);
        if (march && sc)
            launch_pdl(km_sm_applyw_sc<T>, mgrid, mblock, 0, s, g, sc + (TR ? 27 * g.plane : 0), coef, dir, mg.chunk,
                       dinv, U.u[j], w, j, st);
        else if (march)
            launch_pdl(km_sm_applyw<T>, mgrid, mblock, 0, s, g, coef, dir, mg.chunk, dinv, U.u[j], w, j, st);
        else if (!launch_l0st_if<SD, T, LV>(l0st, 0, TR, o0, oc, U.u[j], dinv, nullptr, w, j, steps, st, rb, s))
            launch_pdl(k_sm_applyw<SD, T, LV, TR>, c.grid, c.block, 0, s, o0, oc, dinv, U.u[j], w, j, st);
        if (ev) record_timing_event(ev[2 * j + 1], s);
        launch_dots<T>(N, w, P, j + 1, j, 0, st, rb, s);
        launch_update<T>(N, w, U.u[j + 1], P, j, steps, 0, st, rb, s);
    }
    launch_sm_combine<T>(N, x, dinv, P, steps, zero_init, st, s);
}

template <typename T>
void launch_smooth(int sd, int lvl, const OpL0<T>& o0, const OpLc<T>& oc, bool tr, const T* b, T* x, const T* dinv,
                   Basis<T> U, T* w, T* w2, int steps, bool zero_init, SmState* st, RedBuf rb, cudaStream_t s,
                   cudaEvent_t* ev, const T* sc) {
    if (lvl == 0) {
        ST_SD_DISPATCH(sd, if (tr) smooth_impl<SD, T, 0, true>(o0, oc, b, x, dinv, U, w, w2, steps, zero_init, st, rb, s, ev, sc);
                       else smooth_impl<SD, T, 0, false>(o0, oc, b, x, dinv, U, w, w2, steps, zero_init, st, rb, s, ev, sc));
    } else {
        ST_SD_DISPATCH(sd, if (tr) smooth_impl<SD, T, 1, true>(o0, oc, b, x, dinv, U, w, w2, steps, zero_init, st, rb, s, ev, sc);
                       else smooth_impl<SD, T, 1, false>(o0, oc, b, x, dinv, U, w, w2, steps, zero_init, st, rb, s, ev, sc));
    }
}

// x = (add ? x : 0) + omega D^-1 r, element by element
template <typename T>
__global__ void __launch_bounds__(256) k_jac_update(long long n, T omega, const T* __restrict__ dinv,
                                                    const T* __restrict__ r, T* __restrict__ x, int add) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T v = omega * dinv[i] * r[i];
        x[i] = add ? x[i] + v : v;
    }
}

template <typename T>
void launch_jacobi_smooth(int sd, int lvl, const OpL0<T>& o0, const OpLc<T>& oc, bool tr, const T* b, T* x,
                          const T* dinv, T* r, int sweeps, bool zero_init, T omega, cudaStream_t s) {
    const long long N = (lvl == 0 ? o0.g : oc.g).nnodes;
    const int blocks = (int)std::min<long long>(4LL * 1216, (N + 255) / 256);
    for (int k = 0; k < sweeps; ++k) {
        const bool first = k == 0 && zero_init;
        if (!first) launch_residual<T>(sd, lvl, o0, oc, tr, b, x, r, s);
        note_launch(s);
        launch_pdl(k_jac_update<T>, blocks, 256, 0, s, N, omega, dinv, first ? b : (const T*)r, x, first ? 0 : 1);
    }
}

template <typename T>
void launch_coarse_solve(const double* Ainv, int n, bool tr, const T* b, T* x, cudaStream_t s) {
    note_launch(s);
    if (tr)
        launch_pdl(k_coarse_gemv_t<T>, (n + 127) / 128, 128, 0, s, Ainv, n, b, x);
    else
        launch_pdl(k_coarse_gemv<T>, (n * 32 + 255) / 256, 256, 0, s, Ainv, n, b, x);
}

template <typename TZ>
void launch_fg_apply_dots(int sd, const OpL0<double>& op, bool tr, const TZ* z, TZ* zstore, double* w,
                          double* const* V, int j, FgState* fs, RedBuf rb, cudaStream_t s) {
    note_launch(s);
    if (sd == 2 && op.st_dir) {
        dim3 grid, block;
        const MarchGrid mg = march_grid(op.g, grid, block);
        launch_pdl(km_fg_apply<TZ>, grid, block, 0, s, op.g, op.st_coef[tr ? 1 : 0], op.st_dir, mg.chunk, z, zstore, w);
    } else {
        const void* vecs[3] = {z, zstore, w};
        if (fg_march_usable(sd, op, vecs, 3)) {
            launch_fg_march<TZ>(sd, 0, tr, op, z, zstore, nullptr, w, nullptr, RedBuf{}, s);
        } else {
            const LaunchCfg c = node_cfg(op.g);
            ST_SD_DISPATCH(sd, if (tr) launch_pdl(k_fg_apply<SD, TZ, true>, c.grid, c.block, 0, s, op, z, zstore, w);
                           else launch_pdl(k_fg_apply<SD, TZ, false>, c.grid, c.block, 0, s, op, z, zstore, w));
        }
    }
    Ptrs<double> P{};
    for (int q = 0; q <= j; ++q) P.p[q] = V[q];
    launch_dots<double>(op.g.nnodes, w, P, j + 1, j, 1, fs, rb, s);
}

void launch_fg_update_dots(const Geom& g, double* w, double* const* V, int j, int pass, FgState* fs, RedBuf rb,
                           cudaStream_t s) {
    Ptrs<double> P{};
    for (int q = 0; q <= j; ++q) P.p[q] = V[q];
    launch_update<double>(g.nnodes, w, w, P, j, 0, pass == 0 ? 1 : 2, fs, rb, s);
}

template <typename TZ>
void launch_fg_normalize(const Geom& g, const double* w, double* vnext, TZ* bmg, int j, FgState* fs, cudaStream_t s) {
    note_launch(s);
    (void)j;
    const LaunchCfg c = node_cfg(g);
    launch_pdl(k_fg_normalize<TZ>, c.grid, c.block, 0, s, g, w, vnext, bmg, fs);
}

template <typename TZ>
void launch_fg_update_x_dev(const Geom& g, double* x, TZ* const* Z, int m, FgState* fs, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_fg_backsolve, 1, 32, 0, s, fs, -1);
    Ptrs<TZ> P{};
    for (int q = 0; q < m; ++q) P.p[q] = Z[q];
    launch_fg_combine<TZ>(g.nnodes, x, P, -m, fs, s);  // -m: up to m vectors, the count read on the device
}

template <typename TZ>
void launch_fg_update_x(const Geom& g, double* x, TZ* const* Z, int k, FgState* fs, cudaStream_t s) {
    if (k <= 0) return;
    note_launch(s);
    launch_pdl(k_fg_backsolve, 1, 32, 0, s, fs, k);
    Ptrs<TZ> P{};
    for (int q = 0; q < k; ++q) P.p[q] = Z[q];
    launch_fg_combine<TZ>(g.nnodes, x, P, k, fs, s);
}

void launch_fg_residual(int sd, const OpL0<double>& op, bool tr, const double* f, const double* x, double* r,
                        FgState* fs, RedBuf rb, cudaStream_t s) {
    note_launch(s);
    if (sd == 2 && op.st_dir) {
        dim3 grid, block;
        const MarchGrid mg = march_grid(op.g, grid, block);
        launch_pdl(km_fg_residual, grid, block, 0, s, op.g, op.st_coef[tr ? 1 : 0], op.st_dir, mg.chunk, f, x, r, fs, rb);
        return;
    }
    {
        const void* vecs[3] = {f, x, r};
        if (fg_march_usable(sd, op, vecs, 3)) {
            launch_fg_march<double>(sd, 1, tr, op, x, nullptr, f, r, fs, rb, s);
            return;
        }
    }
    const LaunchCfg c = node_cfg(op.g);
    ST_SD_DISPATCH(sd, if (tr) launch_pdl(k_fg_residual<SD, true>, c.grid, c.block, 0, s, op, f, x, r, fs, rb);
                   else launch_pdl(k_fg_residual<SD, false>, c.grid, c.block, 0, s, op, f, x, r, fs, rb));
}

template <typename TZ>
void launch_fg_start(const Geom& g, double* v0, TZ* bmg, FgState* fs, cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(g);
    launch_pdl(k_fg_start<TZ>, c.grid, c.block, 0, s, g, v0, bmg, fs);
}

void launch_dot64(const Geom& g, const double* a, const double* b, double* out, RedBuf rb, cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(g);
    launch_pdl(k_dot64, c.grid, c.block, 0, s, g, a, b, out, rb);
}

void launch_mask_copy(int sd, const Geom& g, const double* src, double* dst, cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(g);
    ST_SD_DISPATCH(sd, launch_pdl(k_mask_copy<SD>, c.grid, c.block, 0, s, g, src, dst));
}

#define ST_INST_T(T)                                                                                                \
    template void launch_apply_l0<T>(int, const OpL0<T>&, bool, const T*, T*, cudaStream_t);                        \
    template void launch_apply_lc<T>(int, const OpLc<T>&, bool, const T*, T*, cudaStream_t);                        \
    template void launch_diag_l0<T>(int, const OpL0<T>&, T*, bool, cudaStream_t);                                   \
    template void launch_diag_lc<T>(int, const OpLc<T>&, T*, bool, cudaStream_t);                                   \
    template void launch_residual<T>(int, int, const OpL0<T>&, const OpLc<T>&, bool, const T*, const T*, T*,        \
                                     cudaStream_t);                                                                  \
    template void launch_restrict<T>(const Geom&, const Geom&, int, int, const T*, T*, cudaStream_t);               \
    template void launch_prolong<T>(const Geom&, const Geom&, int, int, const T*, T*, cudaStream_t);                \
    template void launch_smooth<T>(int, int, const OpL0<T>&, const OpLc<T>&, bool, const T*, T*, const T*, Basis<T>, \
                                   T*, T*, int, bool, SmState*, RedBuf, cudaStream_t, cudaEvent_t*, const T*);      \
    template void launch_coarse_solve<T>(const double*, int, bool, const T*, T*, cudaStream_t);                     \
    template void launch_jacobi_smooth<T>(int, int, const OpL0<T>&, const OpLc<T>&, bool, const T*, T*, const T*,   \
                                          T*, int, bool, T, cudaStream_t);                                           \
    template void launch_fg_apply_dots<T>(int, const OpL0<double>&, bool, const T*, T*, double*, double* const*,    \
                                          int, FgState*, RedBuf, cudaStream_t);                                      \
    template void launch_fg_normalize<T>(const Geom&, const double*, double*, T*, int, FgState*, cudaStream_t);     \
    template void launch_fg_update_x<T>(const Geom&, double*, T* const*, int, FgState*, cudaStream_t);             \
    template void launch_fg_update_x_dev<T>(const Geom&, double*, T* const*, int, FgState*, cudaStream_t);         \
    template void launch_fg_start<T>(const Geom&, double*, T*, FgState*, cudaStream_t);

ST_INST_T(float)
ST_INST_T(double)

}  // namespace st
