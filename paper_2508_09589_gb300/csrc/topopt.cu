// The topology-optimisation loop of Sec. 3.3 (the nested formulation: each design iteration
// solves the state for the current design), one design iteration per st_topopt_step, all on
// the mesh's device and stream.  The steps are the library's own calls (PDE filter and
// projection of Sec. 3.3.2, st_set_design, the forward and adjoint space-time solves of Sec. 3.2,
// the sensitivities of Sec. 3.3.3, the MMA update) joined by four small element-wise kernels:
// the chain-rule products H'(gamma~) * g, the volume sum of the physical design, the clipped
// copy of the initial design and the largest design change.  Sums are deterministic: one
// partial per block of a fixed grid, added in block order on the host.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "st_mesh.h"

namespace st {
namespace {

constexpr int kToThreads = 256;
constexpr int kToBlocks = 1216;  // 8 waves of 152 SMs; grid-stride loops

int to_blocks(long long n) { return (int)std::min<long long>(kToBlocks, (n + kToThreads - 1) / kToThreads); }

__device__ __forceinline__ void to_block_sum(double v, double* part) {
    __shared__ double sh[kToThreads];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kToThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out = c * a * b (b null: c * a)
__global__ void __launch_bounds__(kToThreads) k_to_scale(long long n, double c, const double* __restrict__ a,
                                                         const double* __restrict__ b, double* __restrict__ out) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        out[j] = b ? c * a[j] * b[j] : c * a[j];
}

// out = in clipped to [0, 1]; part[block] = number of non-finite values seen
__global__ void __launch_bounds__(kToThreads) k_to_clip(long long n, const double* __restrict__ in,
                                                        double* __restrict__ out, double* __restrict__ part) {
    double bad = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double v = in[j];
        if (!isfinite(v)) bad += 1.0;
        out[j] = fmin(fmax(v, 0.0), 1.0);
    }
    to_block_sum(bad, part);
}

__global__ void __launch_bounds__(kToThreads) k_to_sum(long long n, const double* __restrict__ a,
                                                       double* __restrict__ part) {
    double s = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        s += a[j];
    to_block_sum(s, part);
}

__global__ void __launch_bounds__(kToThreads) k_to_maxdiff(long long n, const double* __restrict__ a,
                                                           const double* __restrict__ b, double* __restrict__ part) {
    __shared__ double sh[kToThreads];
    double m = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[j] - b[j]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = kToThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

}  // namespace
}  // namespace st

struct st_topopt {
    st_mesh* mesh = nullptr;
    st::Mesh* mm = nullptr;
    st_topopt_params p{};
    int layout = 0;
    long long n = 0;
    int it = 0;            // design iterations taken
    double phi1 = 0.0;     // objective at the first iteration
    double* base = nullptr;
    double *gamma = nullptr, *gt = nullptr, *gb = nullptr, *dh = nullptr, *tmp = nullptr, *df0 = nullptr,
           *dg1 = nullptr, *gprev = nullptr, *part = nullptr;
    std::vector<double> hpart;
    st_mma* mma = nullptr;

    // launch a partial-sum kernel's result back and combine it (sum or max) in block order
    st_status reduce(int blocks, bool take_max, double& out) {
        cudaStream_t s = mm->stream;
        if (cudaMemcpyAsync(hpart.data(), part, blocks * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return st::fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        double t = 0.0;
        for (int b = 0; b < blocks; ++b) t = take_max ? std::max(t, hpart[b]) : t + hpart[b];
        out = t;
        return ST_OK;
    }
};

extern "C" {

void st_topopt_params_default(st_topopt_params* p) {
    if (!p) return;
    p->vf = 0.3;
    p->r_x = 0.0;
    p->r_t = 0.0;
    p->beta = 32.0;
    p->eta = 0.5;
    p->objective = ST_OBJ_PNORM;
    p->P = 20;
    p->obj_scale = 10.0;
    p->filter_rtol = 1e-10;
    p->filter_max_it = 2000;
    p->warm_start = 1;
    st_mma_params_default(&p->mma);
}

st_status st_topopt_create(st_mesh* m, const st_topopt_params* pin, const double* gamma0, int layout, size_t count,
                           int mem, st_topopt** out) {
    using st::fail;
    if (!out) return fail(ST_ERR_ARG, "null output handle");
    *out = nullptr;
    if (!m || !gamma0) return fail(ST_ERR_ARG, "null argument");
    st_topopt_params p;
    if (pin)
        p = *pin;
    else
        st_topopt_params_default(&p);
    if (!(p.vf > 0 && p.vf < 1)) return fail(ST_ERR_ARG, "volume fraction must be in (0, 1)");
    if (!(p.beta > 0) || !(p.eta > 0 && p.eta < 1)) return fail(ST_ERR_ARG, "beta > 0 and 0 < eta < 1 required");
    if (!(p.obj_scale > 0) || !std::isfinite(p.obj_scale)) return fail(ST_ERR_ARG, "obj_scale must be positive");
    if (p.objective != ST_OBJ_PNORM && p.objective != ST_OBJ_COMPLIANCE) return fail(ST_ERR_ARG, "unknown objective");
    if (p.objective == ST_OBJ_PNORM && (p.P < 1 || p.P > 64)) return fail(ST_ERR_ARG, "p-norm exponent must be in [1, 64]");
    if (!(p.filter_rtol > 0) || p.filter_max_it < 1) return fail(ST_ERR_ARG, "filter rtol and max_it must be positive");
    if (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(ST_ERR_ARG, "unknown memory kind");
    st::Mesh* mm = st::mesh_of(m);
    const st::Geom& g0 = mm->lv[0].g;
    const long long want = layout == ST_DESIGN_EXTRUDED ? g0.sp_elems
                           : layout == ST_DESIGN_SPACETIME ? g0.sp_elems * g0.net
                                                           : -1;
    if (want < 0) return fail(ST_ERR_ARG, "unknown design layout");
    if ((long long)count != want) return fail(ST_ERR_ARG, "count does not match the design layout");
    cudaSetDevice(mm->device);
    st_topopt* h = new st_topopt();
    h->mesh = m;
    h->mm = mm;
    h->p = p;
    h->layout = layout;
    h->n = want;
    st_status r = st_mma_create(h->n, &p.mma, &h->mma);
    if (r != ST_OK) {
        delete h;
        return fail(r, "optimiser parameters or memory");
    }
    const long long n = h->n;
    if (cudaMalloc((void**)&h->base, (8 * n + st::kToBlocks) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        st_mma_destroy(h->mma);
        delete h;
        return fail(ST_ERR_OOM, "design buffers");
    }
    double* q = h->base;
    double** f[] = {&h->gamma, &h->gt, &h->gb, &h->dh, &h->tmp, &h->df0, &h->dg1, &h->gprev};
    for (double** d : f) {
        *d = q;
        q += n;
    }
    h->part = q;
    h->hpart.resize(st::kToBlocks);
    cudaStream_t s = mm->stream;
    auto undo = [&](st_status code, const char* msg) {
        cudaStreamSynchronize(s);
        cudaFree(h->base);
        st_mma_destroy(h->mma);
        delete h;
        return fail(code, msg);
    };
    if (cudaMemcpyAsync(h->tmp, gamma0, n * sizeof(double),
                        mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
        return undo(ST_ERR_CUDA, "copy of the initial design");
    const int blocks = st::to_blocks(n);
    st::k_to_clip<<<blocks, st::kToThreads, 0, s>>>(n, h->tmp, h->gamma, h->part);
    st::note_launch(s);
    double bad = 0.0;
    if (h->reduce(blocks, false, bad) != ST_OK) return undo(ST_ERR_CUDA, "initial design");
    if (bad > 0) return undo(ST_ERR_NUMERIC, "NaN/Inf in the initial design");
    *out = h;
    return ST_OK;
}

st_status st_topopt_destroy(st_topopt* h) {
    if (!h) return ST_OK;
    cudaSetDevice(h->mm->device);
    cudaStreamSynchronize(h->mm->stream);
    cudaFree(h->base);
    st_mma_destroy(h->mma);
    delete h;
    return ST_OK;
}

st_status st_topopt_step(st_topopt* h, const st_source* q, const st_options* o, st_topopt_stats* stats) {
    using st::fail;
    if (!h || !q) return fail(ST_ERR_ARG, "null argument");
    const auto t0 = std::chrono::steady_clock::now();
    st::Mesh* mm = h->mm;
    cudaSetDevice(mm->device);
    cudaStream_t s = mm->stream;
    const long long n = h->n;
    const int blocks = st::to_blocks(n);
    const st_topopt_params& p = h->p;
    st_topopt_stats S{};
    bool short_of_tol = false;
    auto soft = [&](st_status r) {  // a capped solve still yields a usable iterate
        if (r == ST_ERR_NOT_CONVERGED) {
            short_of_tol = true;
            return ST_OK;
        }
        return r;
    };
    int its = 0;
    st_status r;
    // host wall time of a part (every part ends with a stream synchronisation)
    auto since = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
    };
    auto filter = [&](const double* in, double* out) {
        const auto tf = std::chrono::steady_clock::now();
        const st_status fr =
            soft(st::filter(mm, in, out, n, ST_MEM_DEVICE, p.r_x, p.r_t, p.filter_rtol, p.filter_max_it, &its));
        S.filter_its += its;
        S.filter_seconds += since(tf);
        return fr;
    };
    // design chain: gamma~ = F gamma, gamma_bar = H(gamma~), H'(gamma~)
    if ((r = filter(h->gamma, h->gt)) != ST_OK) return r;
    const auto td = std::chrono::steady_clock::now();
    st::launch_heaviside(n, h->gt, h->gb, h->dh, p.beta, p.eta, s);
    if ((r = st_set_design(h->mesh, h->gb, h->layout, n, ST_MEM_DEVICE)) != ST_OK) return r;
    cudaStreamSynchronize(s);
    S.design_seconds = since(td);
    // state, objective and adjoint
    st_options opt;
    st_options_default(&opt);
    if (o) opt = *o;
    opt.warm_start = (p.warm_start && h->it >= 1) ? 1 : 0;
    if ((r = soft(st_solve_forward(h->mesh, q, &opt, &S.forward))) != ST_OK) return r;
    st_objective obj{p.objective, p.P};
    double phi = 0.0;
    if ((r = soft(st_solve_adjoint(h->mesh, &obj, &opt, &phi, &S.adjoint))) != ST_OK) return r;
    if (!std::isfinite(phi) || (h->it == 0 && !(phi > 0)))
        return fail(ST_ERR_NUMERIC, "objective is not finite and positive");
    const double phi1 = h->it == 0 ? phi : h->phi1;
    // d phi / d gamma = F (H' * d phi / d gamma_bar), scaled as MMA sees it
    if ((r = st_sensitivities(h->mesh, h->tmp, n, ST_MEM_DEVICE)) != ST_OK) return r;
    st::k_to_scale<<<blocks, st::kToThreads, 0, s>>>(n, p.obj_scale / phi1, h->dh, h->tmp, h->tmp);
    st::note_launch(s);
    if ((r = filter(h->tmp, h->df0)) != ST_OK) return r;
    // chi = mean(gamma_bar) / v_f - 1 (uniform elements) and d chi / d gamma = F (H' / (v_f N))
    const auto tm = std::chrono::steady_clock::now();
    st::k_to_sum<<<blocks, st::kToThreads, 0, s>>>(n, h->gb, h->part);
    st::note_launch(s);
    double vol = 0.0;
    if ((r = h->reduce(blocks, false, vol)) != ST_OK) return r;
    const double chi = vol / (p.vf * (double)n) - 1.0;
    st::k_to_scale<<<blocks, st::kToThreads, 0, s>>>(n, 1.0 / (p.vf * (double)n), h->dh, nullptr, h->tmp);
    st::note_launch(s);
    S.mma_seconds = since(tm);
    if ((r = filter(h->tmp, h->dg1)) != ST_OK) return r;
    // MMA step on gamma in [0, 1]
    const auto tu = std::chrono::steady_clock::now();
    if (cudaMemcpyAsync(h->gprev, h->gamma, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    double lam = 0.0;
    if ((r = st_mma_update(h->mma, h->it + 1, h->gamma, h->df0, chi, h->dg1, 0.0, 1.0, s, &lam)) != ST_OK)
        return fail(r, "MMA update");
    st::k_to_maxdiff<<<blocks, st::kToThreads, 0, s>>>(n, h->gamma, h->gprev, h->part);
    st::note_launch(s);
    double change = 0.0;
    if ((r = h->reduce(blocks, true, change)) != ST_OK) return r;
    S.mma_seconds += since(tu);
    h->it += 1;
    h->phi1 = phi1;
    S.iteration = h->it;
    S.phi = phi;
    S.chi = chi;
    S.lam = lam;
    S.change = change;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (short_of_tol) return fail(ST_ERR_NOT_CONVERGED, "a solve or filter stopped at its iteration cap");
    return ST_OK;
}

st_status st_topopt_get(st_topopt* h, int which, double* out, size_t count, int mem) {
    using st::fail;
    if (!h || !out) return fail(ST_ERR_ARG, "null argument");
    if ((long long)count != h->n) return fail(ST_ERR_ARG, "count must equal the design size");
    if (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(ST_ERR_ARG, "unknown memory kind");
    const double* src = which == ST_TO_GAMMA         ? h->gamma
                        : which == ST_TO_GAMMA_TILDE ? h->gt
                        : which == ST_TO_GAMMA_BAR   ? h->gb
                        : which == ST_TO_DPHI        ? h->df0
                        : which == ST_TO_DCHI        ? h->dg1
                                                     : nullptr;
    if (!src) return fail(ST_ERR_ARG, "unknown field");
    if (which != ST_TO_GAMMA && h->it == 0) return fail(ST_ERR_STATE, "no design iteration taken yet");
    cudaSetDevice(h->mm->device);
    cudaStream_t s = h->mm->stream;
    if (cudaMemcpyAsync(out, src, count * sizeof(double),
                        mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(ST_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    return ST_OK;
}

}  // extern "C"
