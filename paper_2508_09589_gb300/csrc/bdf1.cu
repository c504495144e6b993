// The reference time-stepping solver of the paper's comparison (Sec. 4): first-order backward
// differences in time on the spatial mesh, with consistent capacity-weighted mass,
//   (M_C + dt K_k) T^{n+1} = M_C T^n + dt F(t_{n+1}),   T^0 = 0,
// the design of slab n at step n, F_i(t) = Q(t) int N_i for the spatially uniform sources and the
// spatial sink prescribed at every step.
//
// The step matrix is the upper-plane block of a one-slab space-time system.  Row a_t = 1 of the
// stabilised time matrices is D_t = (-1, 1) and M_t = dt/6 (1, 2), so with T = 0 on the lower
// plane that block reads C M_x + k dt/3 K_x; with the conductivities tripled it is M_C + dt K_k.
// Each step is therefore solved by the library's own FGMRES and multigrid on a one-slab mesh
// (conductivities x 3, final time dt), on which Algorithm 1 can only coarsen in space: the
// spatial multigrid of the paper's reference solver.  The solve starts from the previous plane.
// One kernel forms the step's right-hand side (the element mass product and the load).
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "st_device.cuh"
#include "st_mesh.h"

namespace st {
namespace {

__device__ __forceinline__ double clip01(double v) { return fmin(fmax(v, 0.0), 1.0); }

// the tensor-product element matrices of one spatial element: mass and stiffness entry (a, b)
template <int SD>
__device__ __forceinline__ void elem_mk(const Geom& g, int a, int b, double& me, double& ke) {
    double mm[3], kk[3];
    for (int d = 0; d < SD; ++d) {
        const bool same = ((a >> d) & 1) == ((b >> d) & 1);
        mm[d] = (same ? 2.0 : 1.0) * g.h[d] / 6.0;
        kk[d] = (same ? 1.0 : -1.0) / g.h[d];
    }
    me = 1.0;
    ke = 0.0;
    for (int d = 0; d < SD; ++d) {
        me *= mm[d];
        double t = kk[d];
        for (int e = 0; e < SD; ++e)
            if (e != d) t *= mm[e];
        ke += t;
    }
}

// b (one-slab node vector): 0 on the lower plane; on the upper plane, at free spatial nodes,
// add_i (may be null) + sum over the node's elements of C_e (M_e x)_i (x may be null) + share,
// share = qdt |e| / 2^SD.  gam is the slab's design (clipped to [0, 1] here).  One thread per
// spatial node.
template <int SD>
__global__ void __launch_bounds__(256) k_bdf1_rhs(Geom g, Simp sm, const double* __restrict__ gam,
                                                  const double* __restrict__ x, const double* __restrict__ add,
                                                  double qdt, double* __restrict__ b) {
    const long long plane = g.plane;
    double vol = 1.0;
    for (int d = 0; d < SD; ++d) vol *= g.h[d];
    const double share = qdt * vol / (double)(1 << SD);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < plane;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % g.nx1);
        const int j = (int)((idx / g.nx1) % g.ny1);
        const int k = SD == 3 ? (int)(idx / ((long long)g.nx1 * g.ny1)) : 0;
        b[idx] = 0.0;
        double v = 0.0;
        if (!sp_dir<SD>(g, i, j, k)) {
            if (add) v = add[idx];
            for (int o = 0; o < (1 << SD); ++o) {
                const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1), ez = SD == 3 ? k - 1 + ((o >> 2) & 1) : 0;
                if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
                if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
                double acc = 0.0;
                if (x) {
                    const long long e = ((long long)ez * g.ney + ey) * g.nex + ex;
                    const double C = sm.C_ins + sm.dC * ipow(clip01(gam[e]), sm.p_c);
                    const int bn = (i - ex) | ((j - ey) << 1) | ((k - ez) << 2);  // the node's corner
                    for (int c = 0; c < (1 << SD); ++c) {
                        double me, ke;
                        elem_mk<SD>(g, bn, c, me, ke);
                        acc += me * x[((long long)(ez + ((c >> 2) & 1)) * g.ny1 + (ey + ((c >> 1) & 1))) * g.nx1 +
                                      (ex + (c & 1))];
                    }
                    acc *= C;
                }
                v += acc + share;
            }
        }
        b[plane + idx] = v;
    }
}

// mean of the 2^(SD+1) nodal values of space-time element (n, e) of a trajectory
template <int SD>
__device__ __forceinline__ double traj_mean(const Geom& g, const double* T, int n, int ex, int ey, int ez) {
    double s = 0.0;
    for (int c = 0; c < (2 << SD); ++c) {
        const int cn = n + ((c >> SD) & 1);
        s += T[(long long)cn * g.plane + ((long long)(ez + ((c >> 2) & 1) * (SD == 3)) * g.ny1 + (ey + ((c >> 1) & 1))) *
                                                g.nx1 + (ex + (c & 1))];
    }
    return s / (double)(2 << SD);
}

constexpr int kB1Threads = 256;
constexpr int kB1Blocks = 1216;

// theta = sum over the space-time elements of T_avg^P: one partial per block
template <int SD>
__global__ void __launch_bounds__(kB1Threads) k_bdf1_theta(Geom g, int nt, const double* __restrict__ T, int P,
                                                           double* __restrict__ part) {
    __shared__ double sh[kB1Threads];
    const long long ne = g.sp_elems * nt;
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ne; q += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(q / g.sp_elems);
        const long long e = q % g.sp_elems;
        const int ex = (int)(e % g.nex), ey = (int)((e / g.nex) % g.ney), ez = SD == 3 ? (int)(e / ((long long)g.nex * g.ney)) : 0;
        s += ipow(traj_mean<SD>(g, T, n, ex, ey, ez), P);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kB1Threads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out = d phi / d T on plane m: sum over the node's space-time elements of
// c T_avg,e^(P-1), c = theta^((1-P)/P) / 2^(SD+1)
template <int SD>
__global__ void __launch_bounds__(256) k_bdf1_pgrad(Geom g, int nt, const double* __restrict__ T, int m, int P,
                                                    double c, double* __restrict__ out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.plane;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % g.nx1);
        const int j = (int)((idx / g.nx1) % g.ny1);
        const int k = SD == 3 ? (int)(idx / ((long long)g.nx1 * g.ny1)) : 0;
        double v = 0.0;
        for (int sb = 0; sb < 2; ++sb) {
            const int n = m - 1 + sb;
            if (n < 0 || n >= nt) continue;
            for (int o = 0; o < (1 << SD); ++o) {
                const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1), ez = SD == 3 ? k - 1 + ((o >> 2) & 1) : 0;
                if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
                if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
                v += c * ipow(traj_mean<SD>(g, T, n, ex, ey, ez), P - 1);
            }
        }
        out[idx] = v;
    }
}

// d phi / d gamma_e = -Lambda^{n+1}_e . (C'_e M_e (T^{n+1} - T^n)_e + dt k'_e K_e T^{n+1}_e) per slab n,
// summed over the slabs for an extruded design (one thread per spatial element, slabs in order)
template <int SD>
__global__ void __launch_bounds__(256) k_bdf1_sens(Geom g, Simp sm, const double* __restrict__ gam, int extruded,
                                                   int nt, double dt, const double* __restrict__ T,
                                                   const double* __restrict__ L, double* __restrict__ out) {
    const int NV = 1 << SD;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.sp_elems;
         e += (long long)gridDim.x * blockDim.x) {
        const int ex = (int)(e % g.nex), ey = (int)((e / g.nex) % g.ney), ez = SD == 3 ? (int)(e / ((long long)g.nex * g.ney)) : 0;
        long long node[8];
        for (int c = 0; c < NV; ++c)
            node[c] = ((long long)(ez + ((c >> 2) & 1)) * g.ny1 + (ey + ((c >> 1) & 1))) * g.nx1 + (ex + (c & 1));
        double acc = 0.0;
        for (int n = 0; n < nt; ++n) {
            const double gm = clip01(gam[(extruded ? 0 : (long long)n * g.sp_elems) + e]);
            const double dC = sm.p_c >= 1 ? sm.dC * sm.p_c * ipow(gm, sm.p_c - 1) : 0.0;
            const double dk = sm.p_k >= 1 ? sm.dk * sm.p_k * ipow(gm, sm.p_k - 1) : 0.0;
            const double* T0 = T + (long long)n * g.plane;
            const double* T1 = T0 + g.plane;
            const double* L1 = L + (long long)(n + 1) * g.plane;
            double v = 0.0;
            for (int a = 0; a < NV; ++a) {
                double mt = 0.0, kt = 0.0;
                for (int b = 0; b < NV; ++b) {
                    double me, ke;
                    elem_mk<SD>(g, a, b, me, ke);
                    mt += me * (T1[node[b]] - T0[node[b]]);
                    kt += ke * T1[node[b]];
                }
                v += L1[node[a]] * (dC * mt + dt * dk * kt);
            }
            if (extruded) {
                acc -= v;
            } else {
                out[(long long)n * g.sp_elems + e] = -v;
            }
        }
        if (extruded) out[e] = acc;
    }
}

}  // namespace
}  // namespace st

struct st_bdf1 {
    st_mesh_desc d{};        // the space-time problem
    st::Mesh* mm = nullptr;  // the one-slab step mesh
    int nt = 0;
    double dt = 0.0;
    long long plane = 0, sp = 0;
    int layout = -1;
    double* gam = nullptr;   // the design (sp or nt * sp values)
    double* traj = nullptr;  // T^0 ... T^nt, plane after plane
    double* lam = nullptr;   // Lambda^0 ... Lambda^nt (allocated by the first adjoint)
    double* work = nullptr;  // one plane of d phi / d T and the block partials
    std::vector<double> hpart;
    bool have_traj = false, have_lam = false;

    const double* slab(int n) const { return layout == ST_DESIGN_SPACETIME ? gam + (long long)n * sp : gam; }
    st::Simp simp() const {
        return st::Simp{d.mat.C_ins, d.mat.C_con - d.mat.C_ins, d.mat.k_ins, d.mat.k_con - d.mat.k_ins, d.mat.p_c,
                        d.mat.p_k};
    }
};

extern "C" {

st_status st_bdf1_create(const st_mesh_desc* d, st_bdf1** out) {
    using st::fail;
    if (!out) return fail(ST_ERR_ARG, "null output handle");
    *out = nullptr;
    if (!d) return fail(ST_ERR_ARG, "null description");
    if (d->n_t < 1 || !(d->tau > 0)) return fail(ST_ERR_ARG, "n_t >= 1 and tau > 0 required");
    st_mesh_desc one = *d;
    one.n_t = 1;
    one.tau = d->tau / d->n_t;
    one.mat.k_ins = 3.0 * d->mat.k_ins;
    one.mat.k_con = 3.0 * d->mat.k_con;
    st::Mesh* mm = nullptr;
    st_status r = st::create_mesh(&one, &mm);
    if (r != ST_OK) {
        delete mm;
        return r;
    }
    st_bdf1* h = new st_bdf1();
    h->d = *d;
    h->mm = mm;
    h->nt = d->n_t;
    h->dt = one.tau;
    h->plane = mm->lv[0].g.plane;
    h->sp = mm->lv[0].g.sp_elems;
    if (cudaMalloc((void**)&h->traj, (size_t)(h->nt + 1) * h->plane * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&h->gam, (size_t)h->nt * h->sp * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->traj);
        delete mm;
        delete h;
        return fail(ST_ERR_OOM, "trajectory and design buffers");
    }
    *out = h;
    return ST_OK;
}

st_status st_bdf1_destroy(st_bdf1* h) {
    if (!h) return ST_OK;
    cudaSetDevice(h->mm->device);
    cudaStreamSynchronize(h->mm->stream);
    cudaFree(h->traj);
    cudaFree(h->gam);
    cudaFree(h->lam);
    cudaFree(h->work);
    delete h->mm;
    delete h;
    return ST_OK;
}

st_status st_bdf1_set_design(st_bdf1* h, const double* gamma, int layout, size_t count, int mem) {
    using st::fail;
    if (!h || !gamma) return fail(ST_ERR_ARG, "null argument");
    const long long want = layout == ST_DESIGN_EXTRUDED ? h->sp : layout == ST_DESIGN_SPACETIME ? h->sp * h->nt : -1;
    if (want < 0) return fail(ST_ERR_ARG, "unknown design layout");
    if ((long long)count != want) return fail(ST_ERR_ARG, "count does not match the design layout");
    if (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(ST_ERR_ARG, "unknown memory kind");
    st::Mesh* mm = h->mm;
    cudaSetDevice(mm->device);
    h->layout = -1;
    h->have_traj = h->have_lam = false;
    if (cudaMemcpyAsync(h->gam, gamma, count * sizeof(double),
                        mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, mm->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(mm->stream) != cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    // an extruded design is the step mesh's design for every step; a space-time design's slab n
    // is set at step n (its first slab here, which also checks that slab's values)
    st_status r = st::set_design(mm, h->gam, ST_DESIGN_EXTRUDED, (size_t)h->sp, ST_MEM_DEVICE);
    if (r != ST_OK) return r;
    h->layout = layout;
    return ST_OK;
}

st_status st_bdf1_forward(st_bdf1* h, const st_source* q, const st_options* o, double* T, size_t count, int mem,
                          st_bdf1_stats* stats) {
    using st::fail;
    if (!h || !q) return fail(ST_ERR_ARG, "null argument");
    if (h->layout < 0) return fail(ST_ERR_STATE, "st_bdf1_set_design must precede st_bdf1_forward");
    if (q->kind != ST_SRC_UNIFORM && q->kind != ST_SRC_SIN_T)
        return fail(ST_ERR_ARG, "the time-stepping reference takes the spatially uniform sources");
    if (!std::isfinite(q->q0) || !std::isfinite(q->a) || !std::isfinite(q->b) || !std::isfinite(q->f))
        return fail(ST_ERR_ARG, "source parameters must be finite");
    if (T && (long long)count != (h->nt + 1) * h->plane) return fail(ST_ERR_ARG, "count must be (n_t + 1) plane nodes");
    if (T && mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(ST_ERR_ARG, "unknown memory kind");
    const auto t0 = std::chrono::steady_clock::now();
    st::Mesh* mm = h->mm;
    cudaSetDevice(mm->device);
    cudaStream_t s = mm->stream;
    st_options opt;
    st_options_default(&opt);
    if (o) opt = *o;
    opt.warm_start = 1;
    h->have_traj = h->have_lam = false;
    st_bdf1_stats S{};
    bool short_of_tol = false;
    const st::Geom& g = mm->lv[0].g;
    const st::Simp sm = h->simp();
    const size_t pb = (size_t)h->plane * sizeof(double);
    if (cudaMemsetAsync(h->traj, 0, pb, s) != cudaSuccess) return fail(ST_ERR_CUDA, "trajectory");
    const int blocks = (int)std::min<long long>(4 * 1216, (h->plane + 255) / 256);
    for (int n = 0; n < h->nt; ++n) {
        st_status r;
        if (h->layout == ST_DESIGN_SPACETIME &&
            (r = st::set_design(mm, h->gam + (long long)n * h->sp, ST_DESIGN_EXTRUDED, (size_t)h->sp,
                                ST_MEM_DEVICE)) != ST_OK)
            return r;
        const double t1 = (n + 1) * h->dt;
        const double Q = q->kind == ST_SRC_SIN_T ? q->q0 * (q->a + q->b * sin(2.0 * M_PI * q->f * t1)) : q->q0;
        const double* Tn = h->traj + (long long)n * h->plane;
        st::note_launch(s);
        const double* gs = h->slab(n);
        if (mm->sd == 2)
            st::k_bdf1_rhs<2><<<blocks, 256, 0, s>>>(g, sm, gs, Tn, nullptr, h->dt * Q, mm->f);
        else
            st::k_bdf1_rhs<3><<<blocks, 256, 0, s>>>(g, sm, gs, Tn, nullptr, h->dt * Q, mm->f);
        if (cudaMemsetAsync(mm->s, 0, pb, s) != cudaSuccess ||
            cudaMemcpyAsync(mm->s + h->plane, Tn, pb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        st_stats ss{};
        r = st::solve(mm, false, &opt, &ss);
        if (r == ST_ERR_NOT_CONVERGED)
            short_of_tol = true;
        else if (r != ST_OK)
            return r;
        S.outer_its += ss.outer_its;
        S.max_outer_its = std::max(S.max_outer_its, ss.outer_its);
        S.max_rel_res = std::max(S.max_rel_res, ss.rel_res);
        S.steps = n + 1;
        if (cudaMemcpyAsync(h->traj + (long long)(n + 1) * h->plane, mm->s + h->plane, pb, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    }
    mm->have_state = false;  // the step mesh's state is one plane of the trajectory, not a solve of its own
    h->have_traj = true;
    h->have_lam = false;
    if (T && cudaMemcpyAsync(T, h->traj, count * sizeof(double),
                             mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (short_of_tol) return fail(ST_ERR_NOT_CONVERGED, "a step solve stopped at max_it");
    return ST_OK;
}

st_status st_bdf1_adjoint(st_bdf1* h, int P, const st_options* o, double* phi, double* Lambda, size_t count, int mem,
                          st_bdf1_stats* stats) {
    using st::fail;
    if (!h) return fail(ST_ERR_ARG, "null argument");
    if (!h->have_traj) return fail(ST_ERR_STATE, "st_bdf1_forward must precede st_bdf1_adjoint");
    if (P < 1 || P > 64) return fail(ST_ERR_ARG, "p-norm exponent must be in [1, 64]");
    if (Lambda && (long long)count != (h->nt + 1) * h->plane)
        return fail(ST_ERR_ARG, "count must be (n_t + 1) plane nodes");
    if (Lambda && mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(ST_ERR_ARG, "unknown memory kind");
    const auto t0 = std::chrono::steady_clock::now();
    st::Mesh* mm = h->mm;
    cudaSetDevice(mm->device);
    cudaStream_t s = mm->stream;
    const size_t pb = (size_t)h->plane * sizeof(double);
    if (!h->lam) {
        if (cudaMalloc((void**)&h->lam, (size_t)(h->nt + 1) * pb) != cudaSuccess ||
            cudaMalloc((void**)&h->work, pb + st::kB1Blocks * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->lam);
            h->lam = nullptr;
            return fail(ST_ERR_OOM, "adjoint trajectory");
        }
        h->hpart.resize(st::kB1Blocks);
    }
    h->have_lam = false;
    st_options opt;
    st_options_default(&opt);
    if (o) opt = *o;
    opt.warm_start = 1;
    const st::Geom& g = mm->lv[0].g;
    const st::Simp sm = h->simp();
    double* G = h->work;
    double* part = h->work + h->plane;
    // theta = sum_e T_avg,e^P over the space-time elements (deterministic block partials)
    const long long ne = g.sp_elems * h->nt;
    const int tb = (int)std::min<long long>(st::kB1Blocks, (ne + st::kB1Threads - 1) / st::kB1Threads);
    st::note_launch(s);
    if (mm->sd == 2)
        st::k_bdf1_theta<2><<<tb, st::kB1Threads, 0, s>>>(g, h->nt, h->traj, P, part);
    else
        st::k_bdf1_theta<3><<<tb, st::kB1Threads, 0, s>>>(g, h->nt, h->traj, P, part);
    if (cudaMemcpyAsync(h->hpart.data(), part, tb * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    double theta = 0.0;
    for (int b = 0; b < tb; ++b) theta += h->hpart[b];
    if (!(theta > 0) || !std::isfinite(theta)) return fail(ST_ERR_NUMERIC, "p-norm of the trajectory is not finite and positive");
    const double phiv = pow(theta, 1.0 / P);
    const double c = pow(theta, (1.0 - P) / P) / (double)(2 << mm->sd);
    st_bdf1_stats S{};
    bool short_of_tol = false;
    const int blocks = (int)std::min<long long>(4 * 1216, (h->plane + 255) / 256);
    if (cudaMemsetAsync(h->lam, 0, pb, s) != cudaSuccess) return fail(ST_ERR_CUDA, "adjoint trajectory");
    for (int m = h->nt; m >= 1; --m) {
        st_status r;
        // A_{m-1} Lambda^m = d phi / d T^m + M_m Lambda^{m+1}
        if (h->layout == ST_DESIGN_SPACETIME &&
            (r = st::set_design(mm, h->slab(m - 1), ST_DESIGN_EXTRUDED, (size_t)h->sp, ST_MEM_DEVICE)) != ST_OK)
            return r;
        const double* Lnext = m < h->nt ? h->lam + (long long)(m + 1) * h->plane : nullptr;
        st::note_launch(s, 2);
        if (mm->sd == 2) {
            st::k_bdf1_pgrad<2><<<blocks, 256, 0, s>>>(g, h->nt, h->traj, m, P, c, G);
            st::k_bdf1_rhs<2><<<blocks, 256, 0, s>>>(g, sm, h->slab(m < h->nt ? m : 0), Lnext, G, 0.0, mm->f);
        } else {
            st::k_bdf1_pgrad<3><<<blocks, 256, 0, s>>>(g, h->nt, h->traj, m, P, c, G);
            st::k_bdf1_rhs<3><<<blocks, 256, 0, s>>>(g, sm, h->slab(m < h->nt ? m : 0), Lnext, G, 0.0, mm->f);
        }
        if (cudaMemsetAsync(mm->s, 0, pb, s) != cudaSuccess ||
            (Lnext ? cudaMemcpyAsync(mm->s + h->plane, Lnext, pb, cudaMemcpyDeviceToDevice, s)
                   : cudaMemsetAsync(mm->s + h->plane, 0, pb, s)) != cudaSuccess)
            return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        st_stats ss{};
        r = st::solve(mm, false, &opt, &ss);
        if (r == ST_ERR_NOT_CONVERGED)
            short_of_tol = true;
        else if (r != ST_OK)
            return r;
        S.outer_its += ss.outer_its;
        S.max_outer_its = std::max(S.max_outer_its, ss.outer_its);
        S.max_rel_res = std::max(S.max_rel_res, ss.rel_res);
        S.steps += 1;
        if (cudaMemcpyAsync(h->lam + (long long)m * h->plane, mm->s + h->plane, pb, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    }
    mm->have_state = false;
    h->have_lam = true;
    if (Lambda && cudaMemcpyAsync(Lambda, h->lam, count * sizeof(double),
                                  mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (phi) *phi = phiv;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (short_of_tol) return fail(ST_ERR_NOT_CONVERGED, "a step solve stopped at max_it");
    return ST_OK;
}

st_status st_bdf1_sensitivities(st_bdf1* h, double* out, size_t count, int mem) {
    using st::fail;
    if (!h || !out) return fail(ST_ERR_ARG, "null argument");
    if (!h->have_lam) return fail(ST_ERR_STATE, "st_bdf1_adjoint must precede st_bdf1_sensitivities");
    const long long want = h->layout == ST_DESIGN_EXTRUDED ? h->sp : h->sp * h->nt;
    if ((long long)count != want) return fail(ST_ERR_ARG, "count must equal the design size");
    if (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(ST_ERR_ARG, "unknown memory kind");
    st::Mesh* mm = h->mm;
    cudaSetDevice(mm->device);
    cudaStream_t s = mm->stream;
    double* dst = out;
    double* tmp = nullptr;
    if (mem == ST_MEM_HOST) {
        if (cudaMalloc((void**)&tmp, count * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ST_ERR_OOM, "sensitivity buffer");
        }
        dst = tmp;
    }
    const st::Geom& g = mm->lv[0].g;
    const int blocks = (int)std::min<long long>(4 * 1216, (h->sp + 255) / 256);
    st::note_launch(s);
    const int ex = h->layout == ST_DESIGN_EXTRUDED ? 1 : 0;
    if (mm->sd == 2)
        st::k_bdf1_sens<2><<<blocks, 256, 0, s>>>(g, h->simp(), h->gam, ex, h->nt, h->dt, h->traj, h->lam, dst);
    else
        st::k_bdf1_sens<3><<<blocks, 256, 0, s>>>(g, h->simp(), h->gam, ex, h->nt, h->dt, h->traj, h->lam, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

}  // extern "C"
