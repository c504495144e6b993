// Method of Moving Asymptotes (Svanberg 1987) with one constraint g1(x) <= 0 (the volume
// constraint of Sec. 3.3.1), the optimiser of Sec. 3.3.3, on the device in FP64.  Per variable:
// the asymptotes of the iteration (the first two at x -/+ s0 span, later ones moved by incr or
// decr as the last two steps kept or flipped their sign, within 0.01 .. 10 span of x), the
// subproblem's bounds alpha = max(x_min, L + 0.1 (x - L), x - move span), beta = min(x_max,
// U - 0.1 (U - x), x + move span), and the convex approximation terms
//   p = (U - x)^2 (1.001 d+ + 0.001 d- + raa / span),  q = (x - L)^2 (0.001 d+ + 1.001 d- + raa / span)
// of the objective and the constraint.  The subproblem is solved through its dual: for a
// multiplier lam the minimiser is x_j = (sqrt(P) L + sqrt(Q) U) / (sqrt(P) + sqrt(Q)) clipped to
// [alpha, beta] with P = p0 + lam p1, Q = q0 + lam q1; lam = 0 when the approximated constraint
// holds there, else its root to 1e-15 relative by doubling and Illinois regula falsi on the host
// (each trial one kernel and a deterministic block-partial sum), capped at the first power of two
// at or above lam_max (the most feasible point).
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "st_internal.h"

namespace st {

namespace {

constexpr int kMmaThreads = 256;
constexpr int kMmaBlocks = 1216;  // 8 waves of 152 SMs; grid-stride loops

struct MmaArrays {
    double *xold1, *xold2, *low, *upp, *alpha, *beta, *p0, *q0, *p1, *q1, *part;
};

__device__ __forceinline__ double mma_x_of(double lam, double L, double U, double a, double b, double p0, double q0,
                                           double p1, double q1) {
    const double sp = sqrt(p0 + lam * p1), sq = sqrt(q0 + lam * q1);
    const double x = (sp * L + sq * U) / (sp + sq);
    return fmin(fmax(x, a), b);
}

// per-block partial sums in a fixed order: thread partials, then a tree in shared memory
__device__ __forceinline__ void block_partial(double v, double* part) {
    __shared__ double sh[kMmaThreads];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kMmaThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kMmaThreads) k_mma_prep(long long n, int it, st_mma_params pr, double xmin,
                                                          double xmax, const double* __restrict__ x,
                                                          const double* __restrict__ df0,
                                                          const double* __restrict__ dg1, MmaArrays a) {
    const double span = xmax - xmin, reg = pr.raa / span;
    double s = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double xj = x[j];
        double L, U;
        if (it <= 2) {
            L = xj - pr.s0 * span;
            U = xj + pr.s0 * span;
        } else {
            const double sgn = (xj - a.xold1[j]) * (a.xold1[j] - a.xold2[j]);
            const double fac = sgn > 0.0 ? pr.incr : (sgn < 0.0 ? pr.decr : 1.0);
            L = fmin(fmax(xj - fac * (a.xold1[j] - a.low[j]), xj - 10.0 * span), xj - 0.01 * span);
            U = fmin(fmax(xj + fac * (a.upp[j] - a.xold1[j]), xj + 0.01 * span), xj + 10.0 * span);
        }
        a.low[j] = L;
        a.upp[j] = U;
        a.alpha[j] = fmax(fmax(xmin, L + 0.1 * (xj - L)), xj - pr.move * span);
        a.beta[j] = fmin(fmin(xmax, U - 0.1 * (U - xj)), xj + pr.move * span);
        const double ux2 = (U - xj) * (U - xj), xl2 = (xj - L) * (xj - L);
        const double d0 = df0[j], d1 = dg1[j];
        const double d0p = fmax(d0, 0.0), d0m = fmax(-d0, 0.0), d1p = fmax(d1, 0.0), d1m = fmax(-d1, 0.0);
        a.p0[j] = ux2 * (1.001 * d0p + 0.001 * d0m + reg);
        a.q0[j] = xl2 * (0.001 * d0p + 1.001 * d0m + reg);
        const double p1 = ux2 * (1.001 * d1p + 0.001 * d1m + reg), q1 = xl2 * (0.001 * d1p + 1.001 * d1m + reg);
        a.p1[j] = p1;
        a.q1[j] = q1;
        s += p1 / (U - xj) + q1 / (xj - L);
    }
    block_partial(s, a.part);
}

__global__ void __launch_bounds__(kMmaThreads) k_mma_g(long long n, double lam, MmaArrays a) {
    double s = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double L = a.low[j], U = a.upp[j];
        const double xs = mma_x_of(lam, L, U, a.alpha[j], a.beta[j], a.p0[j], a.q0[j], a.p1[j], a.q1[j]);
        s += a.p1[j] / (U - xs) + a.q1[j] / (xs - L);
    }
    block_partial(s, a.part);
}

__global__ void __launch_bounds__(kMmaThreads) k_mma_final(long long n, double lam, double* __restrict__ x,
                                                           MmaArrays a) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double xs = mma_x_of(lam, a.low[j], a.upp[j], a.alpha[j], a.beta[j], a.p0[j], a.q0[j], a.p1[j], a.q1[j]);
        a.xold2[j] = a.xold1[j];
        a.xold1[j] = x[j];
        x[j] = xs;
    }
}

}  // namespace
}  // namespace st

struct st_mma {
    long long n = 0;
    int device = 0;
    st_mma_params pr{};
    st::MmaArrays a{};
    double* base = nullptr;
    std::vector<double> part;
};

extern "C" {

void st_mma_params_default(st_mma_params* p) {
    if (!p) return;
    p->s0 = 0.05;
    p->incr = 1.2;
    p->decr = 0.7;
    p->move = 0.2;
    p->raa = 1e-5;
    p->lam_max = 1e40;
}

st_status st_mma_create(long long n, const st_mma_params* p, st_mma** out) {
    if (!out || n < 1) return ST_ERR_ARG;
    *out = nullptr;
    st_mma* h = new st_mma();
    h->n = n;
    if (p)
        h->pr = *p;
    else
        st_mma_params_default(&h->pr);
    if (!(h->pr.s0 > 0) || !(h->pr.incr >= 1) || !(h->pr.decr > 0 && h->pr.decr <= 1) || !(h->pr.move > 0) ||
        !(h->pr.raa > 0) || !(h->pr.lam_max > 1) || !std::isfinite(h->pr.lam_max) || !std::isfinite(h->pr.incr) ||
        !std::isfinite(h->pr.s0) || !std::isfinite(h->pr.move) || !std::isfinite(h->pr.raa)) {
        delete h;
        return ST_ERR_ARG;
    }
    cudaGetDevice(&h->device);
    const long long bytes = (10 * n + st::kMmaBlocks) * (long long)sizeof(double);
    if (cudaMalloc((void**)&h->base, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return ST_ERR_OOM;
    }
    cudaMemset(h->base, 0, bytes);
    double* q = h->base;
    double** f[] = {&h->a.xold1, &h->a.xold2, &h->a.low, &h->a.upp, &h->a.alpha,
                    &h->a.beta, &h->a.p0, &h->a.q0, &h->a.p1, &h->a.q1};
    for (double** d : f) {
        *d = q;
        q += n;
    }
    h->a.part = q;
    h->part.resize(st::kMmaBlocks);
    *out = h;
    return ST_OK;
}

st_status st_mma_destroy(st_mma* h) {
    if (!h) return ST_OK;
    cudaSetDevice(h->device);
    cudaFree(h->base);
    delete h;
    return ST_OK;
}

st_status st_mma_update(st_mma* h, int it, double* x, const double* df0, double g1, const double* dg1, double xmin,
                        double xmax, void* stream, double* lam_out) {
    if (!h || !x || !df0 || !dg1 || it < 1 || !(xmax > xmin) || !std::isfinite(g1)) return ST_ERR_ARG;
    cudaSetDevice(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = h->n;
    const int blocks = (int)std::min<long long>(st::kMmaBlocks, (n + st::kMmaThreads - 1) / st::kMmaThreads);
    auto sum_part = [&](double& out) -> bool {
        if (cudaMemcpyAsync(h->part.data(), h->a.part, blocks * sizeof(double), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return false;
        double t = 0.0;
        for (int b = 0; b < blocks; ++b) t += h->part[b];
        out = t;
        return true;
    };
    st::k_mma_prep<<<blocks, st::kMmaThreads, 0, s>>>(n, it, h->pr, xmin, xmax, x, df0, dg1, h->a);
    st::note_launch(s);
    double s1 = 0.0;
    if (!sum_part(s1)) return ST_ERR_CUDA;
    const double r1 = g1 - s1;
    auto g_of = [&](double lam, double& g) -> bool {
        st::k_mma_g<<<blocks, st::kMmaThreads, 0, s>>>(n, lam, h->a);
        st::note_launch(s);
        double t = 0.0;
        if (!sum_part(t)) return false;
        g = t + r1;
        return true;
    };
    double lam = 0.0, g = 0.0;
    if (!g_of(0.0, g)) return ST_ERR_CUDA;
    if (g > 0.0) {
        // the bracket: powers of two from 1 up to the first at or above lam_max.  When the
        // approximated constraint still fails there, the root search would end at that power
        // (g decreases in lam), so it is tested first and taken at once.
        double cap = 1.0;
        while (cap < h->pr.lam_max) cap *= 2.0;
        double gcap = 0.0;
        if (!g_of(cap, gcap)) return ST_ERR_CUDA;
        if (gcap > 0.0) {
            lam = cap;
        } else {
            double lo = 0.0, hi = 1.0, glo = g, ghi = 0.0;
            for (;;) {
                if (!g_of(hi, ghi)) return ST_ERR_CUDA;
                if (!(ghi > 0.0)) break;
                lo = hi;
                glo = ghi;
                hi *= 2.0;
            }
            // root of g in (lo, hi] to 1e-15 relative: regula falsi with the Illinois
            // modification (the value kept at an end twice in a row is halved), falling back to
            // the midpoint when the secant point leaves the bracket
            int side = 0;
            for (int k = 0; k < 400 && hi - lo > 1e-15 * hi; ++k) {
                double mid = hi - ghi * (hi - lo) / (ghi - glo);
                if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double gm = 0.0;
                if (!g_of(mid, gm)) return ST_ERR_CUDA;
                if (gm > 0.0) {
                    lo = mid;
                    glo = gm;
                    if (side < 0) ghi *= 0.5;
                    side = -1;
                } else {
                    hi = mid;
                    ghi = gm;
                    if (gm == 0.0) break;
                    if (side > 0) glo *= 0.5;
                    side = 1;
                }
            }
            lam = hi;
        }
    }
    st::k_mma_final<<<blocks, st::kMmaThreads, 0, s>>>(n, lam, x, h->a);
    st::note_launch(s);
    if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
    if (lam_out) *lam_out = lam;
    return ST_OK;
}

}  // extern "C"
