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

#include "st_device.cuh"
#include "st_mesh.h"

namespace st {
namespace {

// b (one-slab node vector): 0 on the lower plane; on the upper plane, at free spatial nodes,
// sum over the node's elements of C_e (M_e T^n)_i + qdt |e| / 2^SD.  One thread per spatial node.
template <int SD>
__global__ void __launch_bounds__(256) k_bdf1_rhs(Geom g, Simp sm, const double* __restrict__ gam,
                                                  const double* __restrict__ Tn, double qdt,
                                                  double* __restrict__ b) {
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
            for (int o = 0; o < (1 << SD); ++o) {
                const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1), ez = SD == 3 ? k - 1 + ((o >> 2) & 1) : 0;
                if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
                if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
                const long long e = ((long long)ez * g.ney + ey) * g.nex + ex;
                const double C = sm.C_ins + sm.dC * ipow(gam[e], sm.p_c);
                const int bx = i - ex, by = j - ey, bz = k - ez;  // the node's corner in the element
                double acc = 0.0;
                for (int c = 0; c < (1 << SD); ++c) {
                    const int cx = c & 1, cy = (c >> 1) & 1, cz = SD == 3 ? (c >> 2) & 1 : 0;
                    double w = (cx == bx ? 2.0 : 1.0) * g.h[0] / 6.0 * (cy == by ? 2.0 : 1.0) * g.h[1] / 6.0;
                    if (SD == 3) w *= (cz == bz ? 2.0 : 1.0) * g.h[2] / 6.0;
                    acc += w * Tn[((long long)(ez + cz) * g.ny1 + (ey + cy)) * g.nx1 + (ex + cx)];
                }
                v += C * acc + share;
            }
        }
        b[plane + idx] = v;
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
    st_bdf1_stats S{};
    bool short_of_tol = false;
    const st::Geom& g = mm->lv[0].g;
    st::Simp sm{h->d.mat.C_ins, h->d.mat.C_con - h->d.mat.C_ins, h->d.mat.k_ins, h->d.mat.k_con - h->d.mat.k_ins,
                h->d.mat.p_c, h->d.mat.p_k};
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
        if (mm->sd == 2)
            st::k_bdf1_rhs<2><<<blocks, 256, 0, s>>>(g, sm, mm->g64, Tn, h->dt * Q, mm->f);
        else
            st::k_bdf1_rhs<3><<<blocks, 256, 0, s>>>(g, sm, mm->g64, Tn, h->dt * Q, mm->f);
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
    if (T && cudaMemcpyAsync(T, h->traj, count * sizeof(double),
                             mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (short_of_tol) return fail(ST_ERR_NOT_CONVERGED, "a step solve stopped at max_it");
    return ST_OK;
}

}  // extern "C"
