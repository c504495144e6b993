// Host side of the space-time solver: mesh and hierarchy (Algorithm 1), design set-up
// (Galerkin coarse operators, Jacobi diagonals, coarsest inverse), the FP64 flexible
// GMRES with the multigrid V-cycle preconditioner (arXiv 2508.09589, Sec. 3.2), the
// adjoint solve and sensitivities (Sec. 3.3.3), and the C ABI declared in include/st.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <string>
#include <vector>

#include "st_internal.h"
#include "st_mesh.h"

namespace st {

thread_local std::string g_last_error;
thread_local const char* g_last_error_static = nullptr;

st_status fail(st_status code, const std::string& msg) {
    g_last_error = msg;
    g_last_error_static = nullptr;
    return code;
}

st_status set_c_error(st_status code, const char* msg) {
    g_last_error_static = msg;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA,               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

#define CKS(call)                      \
    do {                               \
        st_status s_ = (call);         \
        if (s_ != ST_OK) return s_;    \
    } while (0)

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------- device memory
st_status Mesh::alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ST_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    allocs.push_back(*p);
    alloc_sizes.push_back(bytes);
    bytes_held += (long long)bytes;
    return ST_OK;
}

void Mesh::release(void* p) {
    if (!p) return;
    for (size_t q = 0; q < allocs.size(); ++q)
        if (allocs[q] == p) {
            cudaFree(p);
            bytes_held -= (long long)alloc_sizes[q];
            allocs.erase(allocs.begin() + q);
            alloc_sizes.erase(alloc_sizes.begin() + q);
            return;
        }
}

Mesh::~Mesh() {
    if (device >= 0) cudaSetDevice(device);
    if (stream) cudaStreamSynchronize(stream);
    if (level_timing && tcycles > 0) {
        fprintf(stderr, "[st level timing] %d V-cycles, ms per V-cycle: level: pre-smooth, residual+restrict, prolong+post-smooth\n", tcycles);
        for (size_t l = 0; l < lv.size(); ++l)
            fprintf(stderr, "  L%zu (%lld nodes): %.3f %.3f %.3f\n", l, lv[l].g.nnodes, tacc[l * 3] / tcycles,
                    tacc[l * 3 + 1] / tcycles, tacc[l * 3 + 2] / tcycles);
    }
    for (cudaEvent_t e : tev) cudaEventDestroy(e);
    for (cudaEvent_t e : at_ev)
        if (e) cudaEventDestroy(e);
    if (vt_trace) {
        std::vector<unsigned long long> t(4096);
        cudaMemcpy(t.data(), vt_trace, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        fprintf(stderr, "[st vtail trace] ns between barriers of the last tail launch:");
        for (int q = 1; q < 4096 && t[q] > t[0]; ++q) fprintf(stderr, " %llu", t[q] - t[q - 1]);
        fprintf(stderr, "\n");
        cudaFree(vt_trace);
    }
    drop_graphs();
    for (void* p : allocs) cudaFree(p);
    if (h_fg) cudaFreeHost(h_fg);
    if (own_stream && own) cudaStreamDestroy(own);
}

void Mesh::timer_collect() {
    if (!at_pending) return;
    at_pending = false;
    for (int sw = 0; sw < 2; ++sw)
        for (int j = 0; j < at_steps; ++j) {
            float ms = 0.f;
            cudaEvent_t* e = at_ev + sw * 2 * kMaxSmooth + 2 * j;
            if (cudaEventElapsedTime(&ms, e[0], e[1]) == cudaSuccess) {
                at_ms += ms;
                ++at_launches;
            } else {
                cudaGetLastError();
            }
        }
}

void Mesh::drop_graphs() {
    for (int q = 0; q < 4; ++q) {
        if (gexec[q]) cudaGraphExecDestroy(gexec[q]);
        gexec[q] = nullptr;
    }
}

// ---------------------------------------------------------------- geometry
static void patch_range(int n, double w, int& lo, int& hi) {
    lo = n + 1;
    hi = -1;
    for (int j = 0; j <= n; ++j)
        if (fabs(2.0 * j - n) <= w * n + 1e-9) {
            lo = std::min(lo, j);
            hi = std::max(hi, j);
        }
}

static Geom make_geom(const st_mesh_desc& d, const int n[3], int nt, const double h[3], double dt) {
    Geom g{};
    const int sd = d.ndim_space;
    g.nex = n[0];
    g.ney = n[1];
    g.nez = sd == 3 ? n[2] : 1;
    g.net = nt;
    g.nx1 = g.nex + 1;
    g.ny1 = g.ney + 1;
    g.nz1 = sd == 3 ? g.nez + 1 : 1;
    g.nt1 = nt + 1;
    g.plane = (long long)g.nx1 * g.ny1 * g.nz1;
    g.nnodes = g.plane * g.nt1;
    g.sp_elems = (long long)g.nex * g.ney * g.nez;
    for (int q = 0; q < 3; ++q) g.h[q] = h[q];
    g.dt = dt;
    g.bc = d.bc;
    g.face = d.bc == ST_BC_PATCH_BOTTOM ? 1 : 0;
    for (int q = 0; q < 3; ++q) {
        g.plo[q] = 0;
        g.phi[q] = -1;
    }
    for (int q = 0; q < sd; ++q) patch_range(n[q], d.bc_width, g.plo[q], g.phi[q]);
    g.march_blocks = d.march_blocks;
    return g;
}

// Algorithm 1: lambda = D_eff dt / dx^2 (dx: smallest spatial size); coarsen time when
// lambda < lambda_crit, else space; fall back to the other axis when the chosen one cannot
// be halved; stop at max_levels or once a level has at most coarse_dof_cap nodes.
static st_status build_levels(const st_mesh_desc& d, std::vector<LevelH>& lv) {
    const int sd = d.ndim_space;
    const double Deff = sqrt(d.mat.k_con * d.mat.k_ins / (d.mat.C_con * d.mat.C_ins));
    int n[3] = {d.n[0], d.n[1], sd == 3 ? d.n[2] : 1};
    int nt = d.n_t;
    double h[3] = {d.ext[0] / d.n[0], d.ext[1] / d.n[1], sd == 3 ? d.ext[2] / d.n[2] : 1.0};
    double dt = d.tau / d.n_t;
    lv.clear();
    for (;;) {
        LevelH L;
        L.g = make_geom(d, n, nt, h, dt);
        const bool done = (d.max_levels > 0 && (int)lv.size() + 1 >= d.max_levels) ||
                          L.g.nnodes <= d.coarse_dof_cap || (int)lv.size() + 1 >= kMaxLevels;
        bool can_s = true;
        for (int q = 0; q < sd; ++q) can_s = can_s && n[q] % 2 == 0 && n[q] >= 4;
        const bool can_t = nt % 2 == 0 && nt >= 2;
        int kind = -1;
        if (d.coarsening == ST_COARSEN_FULL) {
            kind = (can_s && can_t) ? 2 : -1;
        } else {
            double hmin = h[0];
            for (int q = 1; q < sd; ++q) hmin = std::min(hmin, h[q]);
            const double lam = Deff * dt / (hmin * hmin);
            kind = lam < d.lambda_crit ? 1 : 0;
            if (kind == 1 && !can_t) kind = can_s ? 0 : -1;
            else if (kind == 0 && !can_s) kind = can_t ? 1 : -1;
        }
        if (done || kind < 0) {
            L.to_next = -1;
            lv.push_back(L);
            break;
        }
        L.to_next = kind;
        lv.push_back(L);
        if (kind == 0 || kind == 2)
            for (int q = 0; q < sd; ++q) {
                n[q] /= 2;
                h[q] *= 2;
            }
        if (kind == 1 || kind == 2) {
            nt /= 2;
            dt *= 2;
        }
    }
    return ST_OK;
}

static st_status build_hierarchy(Mesh* m) {
    CKS(build_levels(m->desc, m->lv));
    const long long nc = m->lv.back().g.nnodes;
    m->coarse_iter = m->desc.coarse_solver == ST_COARSE_GMRES ||
                     (m->desc.coarse_solver == ST_COARSE_AUTO && nc > kMaxCoarse);
    if (nc > kMaxCoarse && !m->coarse_iter)
        return fail(ST_ERR_ARG, "coarsest level has " + std::to_string(nc) + " nodes (> " +
                                    std::to_string(kMaxCoarse) +
                                    "): the element counts cannot be halved far enough for the dense coarsest solve; "
                                    "use counts with more factors of 2 or the Jacobi-GMRES coarsest solver");
    return ST_OK;
}

template <typename T>
OpL0<T> Mesh::op0() const {
    OpL0<T> o{};
    o.g = lv[0].g;
    o.g64 = g64;
    o.g16 = g16;
    o.tc = layout == ST_DESIGN_EXTRUDED ? 1 : 0;
    o.simp.C_ins = desc.mat.C_ins;
    o.simp.dC = desc.mat.C_con - desc.mat.C_ins;
    o.simp.k_ins = desc.mat.k_ins;
    o.simp.dk = desc.mat.k_con - desc.mat.k_ins;
    o.simp.p_c = desc.mat.p_c;
    o.simp.p_k = desc.mat.p_k;
    const int NS = 1 << sd;
    for (int mb = 0; mb < 8; ++mb) {
        double mx = 1.0, kx = 0.0;
        if (mb < NS) {
            for (int dd = 0; dd < sd; ++dd) mx *= ((mb >> dd) & 1) ? o.g.h[dd] / 6.0 : o.g.h[dd] / 3.0;
            for (int dd = 0; dd < sd; ++dd) {
                double t = ((mb >> dd) & 1) ? -1.0 / o.g.h[dd] : 1.0 / o.g.h[dd];
                for (int e = 0; e < sd; ++e)
                    if (e != dd) t *= ((mb >> e) & 1) ? o.g.h[e] / 6.0 : o.g.h[e] / 3.0;
                kx += t;
            }
        } else {
            mx = 0.0;
        }
        o.mxd[mb] = (T)mx;
        o.kxd[mb] = (T)kx;
    }
    o.dt6 = (T)(o.g.dt / 6.0);
    if (lv[0].sdir) {
        const long long half = 4LL * 27 * lv[0].g.plane;
        const T* base;
        if constexpr (sizeof(T) == 4)
            base = lv[0].st32;
        else
            base = lv[0].st64;
        o.st_coef[0] = base;
        o.st_coef[1] = base + half;
        o.st_dir = lv[0].sdir;
    }
    return o;
}

template <>
OpLc<double> Mesh::opc<double>(int l) const {
    OpLc<double> o{};
    o.g = lv[l].g;
    o.elem = l > 0 ? lv[l].e64 : nullptr;
    o.tc = layout == ST_DESIGN_EXTRUDED ? 1 : 0;
    if (l > 0 && lv[l].sdir) {
        o.st_coef[0] = lv[l].st64;
        o.st_coef[1] = lv[l].st64 + 4LL * 27 * lv[l].g.plane;
        o.st_dir = lv[l].sdir;
    }
    return o;
}

template <>
OpLc<float> Mesh::opc<float>(int l) const {
    OpLc<float> o{};
    o.g = lv[l].g;
    o.elem = l > 0 ? lv[l].e32 : nullptr;
    o.tc = layout == ST_DESIGN_EXTRUDED ? 1 : 0;
    if (l > 0 && lv[l].sdir) {
        o.st_coef[0] = lv[l].st32;
        o.st_coef[1] = lv[l].st32 + 4LL * 27 * lv[l].g.plane;
        o.st_dir = lv[l].sdir;
    }
    if (l > 0 && lv[l].x3st) {
        o.x3st = lv[l].x3st;
        for (int q = 0; q < 8; ++q) o.x3tw[q] = lv[l].x3tw[q];
    }
    if (l > 0) o.x2blk = lv[l].x2blk;
    return o;
}

// ---------------------------------------------------------------- creation
st_status validate_desc(const st_mesh_desc* d) {
    if (!d) return fail(ST_ERR_ARG, "null argument");
    const int sd = d->ndim_space;
    if (sd != 2 && sd != 3) return fail(ST_ERR_ARG, "ndim_space must be 2 or 3");
    for (int q = 0; q < sd; ++q)
        if (d->n[q] < 1 || d->ext[q] <= 0) return fail(ST_ERR_ARG, "spatial element counts and extents must be positive");
    if (d->n_t < 1 || d->tau <= 0) return fail(ST_ERR_ARG, "n_t and tau must be positive");
    if (d->mat.p_c < 1 || d->mat.p_k < 1 || d->mat.p_c > 16 || d->mat.p_k > 16)
        return fail(ST_ERR_ARG, "SIMP powers must be integers in [1, 16]");
    if (!(d->mat.C_ins > 0 && d->mat.C_con > 0 && d->mat.k_ins > 0 && d->mat.k_con > 0))
        return fail(ST_ERR_ARG, "material constants must be positive");
    if (d->bc < 0 || d->bc > 3) return fail(ST_ERR_ARG, "unknown boundary-condition kind");
    if (d->march_blocks < 0 || d->march_blocks > kMaxBlocks)
        return fail(ST_ERR_ARG, "march_blocks must be in [0, " + std::to_string(kMaxBlocks) + "]");
    if (d->coarse_solver < ST_COARSE_AUTO || d->coarse_solver > ST_COARSE_GMRES)
        return fail(ST_ERR_ARG, "unknown coarse_solver");
    if (d->coarse_max_it < 0 || d->coarse_rtol < 0 || !(d->coarse_rtol < 1))
        return fail(ST_ERR_ARG, "coarse_max_it must be >= 0 and coarse_rtol in [0, 1)");
    if (d->smoother != ST_SMOOTH_GMRES && d->smoother != ST_SMOOTH_JACOBI) return fail(ST_ERR_ARG, "unknown smoother");
    if (d->smoother == ST_SMOOTH_JACOBI && !(d->smoother_omega > 0 && d->smoother_omega <= 1))
        return fail(ST_ERR_ARG, "Jacobi damping must be in (0, 1]");
    if (d->coarse_dof_cap < 1 || d->coarse_dof_cap > kMaxCoarse)
        return fail(ST_ERR_ARG, "coarse_dof_cap must be in [1, " + std::to_string(kMaxCoarse) + "]");
    long long nn = d->n_t + 1;
    for (int q = 0; q < sd; ++q) nn *= d->n[q] + 1;
    if (nn > (1LL << 31) - 1) return fail(ST_ERR_ARG, "more than 2^31 - 1 nodes");
    // one time plane's (x, y) node tiles must fit the partial-sum buffer of the reducing kernels
    const long long tiles = (long long)((d->n[0] + 1 + 31) / 32) * ((d->n[1] + 1 + 7) / 8);
    if (tiles > kMaxBlocks) return fail(ST_ERR_ARG, "x-y plane too large (more than 4096 32x8 node tiles)");
    return ST_OK;
}

st_status plan_hierarchy(const st_mesh_desc* d, st_level_info* out, int max_out, int* n_levels) {
    CKS(validate_desc(d));
    std::vector<LevelH> lv;
    CKS(build_levels(*d, lv));
    if (n_levels) *n_levels = (int)lv.size();
    for (int l = 0; l < (int)lv.size() && l < max_out && out; ++l) {
        const Geom& g = lv[l].g;
        st_level_info& li = out[l];
        li.n[0] = g.nex;
        li.n[1] = g.ney;
        li.n[2] = d->ndim_space == 3 ? g.nez : 0;
        li.n_t = g.net;
        li.n_nodes = g.nnodes;
        li.to_next = lv[l].to_next;
        for (int q = 0; q < 3; ++q) li.h[q] = g.h[q];
        li.dt = g.dt;
    }
    return ST_OK;
}

st_status create_mesh(const st_mesh_desc* d, Mesh** out) {
    if (!d || !out) return fail(ST_ERR_ARG, "null argument");
    *out = nullptr;
    CKS(validate_desc(d));
    const int sd = d->ndim_space;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ST_ERR_CUDA, "no CUDA device available");
    }
    if (d->device < 0 || d->device >= ndev) return fail(ST_ERR_ARG, "device ordinal out of range");
    Mesh* m = new Mesh();
    m->desc = *d;
    m->sd = sd;
    m->device = d->device;
    cudaSetDevice(m->device);
    st_status st = build_hierarchy(m);
    if (st != ST_OK) {
        delete m;
        return st;
    }
    if (cudaStreamCreateWithFlags(&m->own, cudaStreamNonBlocking) != cudaSuccess) {
        delete m;
        return fail(ST_ERR_CUDA, "stream creation failed");
    }
    m->own_stream = true;
    m->stream = m->own;
    if (const char* e = getenv("ST_VTAIL_NODES")) m->vt_max_nodes = atoll(e);
    if (const char* e = getenv("ST_VTAIL_SPIN_LIMIT")) {
        const long long v = atoll(e);  // a test shortens the barrier waits to make them give up
        if (v >= 1 && v <= (1LL << 24)) m->vt_spin_limit = (unsigned)v;
    }
    if (const char* e = getenv("ST_LEVEL_TIMING")) m->level_timing = atoi(e) != 0;
    if (const char* e = getenv("ST_VTAIL_TRACE"))
        if (atoi(e) != 0) cudaMalloc((void**)&m->vt_trace, 4096 * sizeof(unsigned long long));
    if (m->level_timing) {
        m->tev.resize(m->lv.size() * 4);
        for (auto& e : m->tev) cudaEventCreate(&e);
        m->tacc.assign(m->lv.size() * 3, 0.0);
    }
    m->vt_first = -1;
    if (m->vt_max_nodes > 0 && !m->coarse_iter)
        for (int l = 0; l < (int)m->lv.size(); ++l)
            if (m->lv[l].g.nnodes <= m->vt_max_nodes && l < (int)m->lv.size() - 1) {
                m->vt_first = l;
                break;
            }
    const long long N = m->lv[0].g.nnodes;
    st = ST_OK;
    auto A = [&](void** p, size_t b) {
        if (st == ST_OK) st = m->alloc(p, b);
    };
    A((void**)&m->f, N * sizeof(double));
    A((void**)&m->s, N * sizeof(double));
    A((void**)&m->lam, N * sizeof(double));
    A((void**)&m->adjrhs, N * sizeof(double));
    A((void**)&m->fg_w, N * sizeof(double));
    A((void**)&m->d_fg, sizeof(FgState));
    A((void**)&m->d_sm, sizeof(SmState));
    A((void**)&m->rb.part, sizeof(double) * kMaxBlocks * kRedQ);
    A((void**)&m->rb.counter, sizeof(unsigned) * 4);
    A((void**)&m->d_scalar, sizeof(double) * 8);
    A((void**)&m->d_err, sizeof(int) * 4);
    A((void**)&m->d_bar, sizeof(unsigned) * 4);
    A((void**)&m->vt_part, sizeof(double) * 2 * kMaxBlocks * kRedQ);
    const long long nc = m->lv.back().g.nnodes;
    if (m->coarse_iter) {
        const int cmax = m->desc.coarse_max_it > 0 ? m->desc.coarse_max_it : 200;
        m->cg_m = std::min(kMaxSmooth, cmax);
        m->cg_cycles = (cmax + m->cg_m - 1) / m->cg_m;
        A((void**)&m->cg_b, nc * sizeof(double));
        A((void**)&m->cg_x, nc * sizeof(double));
        A((void**)&m->cg_dinv, nc * sizeof(double));
        A((void**)&m->cg_w, nc * sizeof(double));
        A((void**)&m->cg_w2, nc * sizeof(double));
        for (int q = 0; q <= m->cg_m; ++q) A((void**)&m->cg_U.u[q], nc * sizeof(double));
        A((void**)&m->d_smc, sizeof(SmState));
    } else {
        A((void**)&m->Ainv, nc * nc * sizeof(double));
        A((void**)&m->Awork, nc * nc * sizeof(double));
        A((void**)&m->pinv, (nc + 1) * sizeof(double));
        A((void**)&m->gjpr, 8 * (size_t)nc * sizeof(double));
    }
    if (st == ST_OK && cudaMallocHost((void**)&m->h_fg, sizeof(FgState)) != cudaSuccess) {
        cudaGetLastError();
        st = fail(ST_ERR_OOM, "pinned host allocation failed");
    }
    if (st != ST_OK) {
        delete m;
        return st;
    }
    cudaMemsetAsync(m->rb.counter, 0, sizeof(unsigned) * 4, m->stream);
    cudaMemsetAsync(m->d_sm, 0, sizeof(SmState), m->stream);
    if (m->d_smc) cudaMemsetAsync(m->d_smc, 0, sizeof(SmState), m->stream);
    cudaMemsetAsync(m->s, 0, N * sizeof(double), m->stream);
    cudaMemsetAsync(m->lam, 0, N * sizeof(double), m->stream);
    cudaMemsetAsync(m->f, 0, N * sizeof(double), m->stream);
    cudaMemsetAsync(m->d_err, 0, sizeof(int) * 4, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        delete m;
        return fail(ST_ERR_CUDA, "initialisation failed");
    }
    *out = m;
    return ST_OK;
}

// ---------------------------------------------------------------- design set-up
st_status Mesh::ensure_level_storage() {
    const int tc = layout == ST_DESIGN_EXTRUDED ? 1 : 0;
    if (storage_tc == tc) return ST_OK;
    drop_graphs();
    for (size_t l = 0; l < lv.size(); ++l) {
        release(lv[l].e64);
        release(lv[l].e32);
        release(lv[l].st64);
        release(lv[l].st32);
        release(lv[l].sdir);
        release(lv[l].x3st);
        lv[l].x3st = nullptr;
        release(lv[l].x2blk);
        lv[l].x2blk = nullptr;
        lv[l].e64 = nullptr;
        lv[l].e32 = nullptr;
        lv[l].st64 = nullptr;
        lv[l].st32 = nullptr;
        lv[l].sdir = nullptr;
    }
    for (size_t l = 1; l < lv.size(); ++l) {
        const Geom& g = lv[l].g;
        lv[l].nstore = tc ? 2 * g.sp_elems : (long long)g.net * g.sp_elems;
        CKS(alloc((void**)&lv[l].e64, lv[l].nstore * nvals(sd) * sizeof(double)));
        CKS(alloc((void**)&lv[l].e32, lv[l].nstore * nvals(sd) * sizeof(float)));
    }
    if (tc && sd == 2) {
        for (size_t l = 0; l < lv.size(); ++l) {
            const long long P = lv[l].g.plane;
            CKS(alloc((void**)&lv[l].st64, 8LL * 27 * P * sizeof(double)));
            CKS(alloc((void**)&lv[l].st32, 8LL * 27 * P * sizeof(float)));
            CKS(alloc((void**)&lv[l].sdir, P));
        }
    }
    if (tc && sd == 3) {
        for (size_t l = 1; l < lv.size(); ++l)
            if (lv[l].g.net >= 2) CKS(alloc((void**)&lv[l].x3st, 54LL * lv[l].g.plane * sizeof(float)));
    }
    if (!tc && sd == 2) {  // levels reached from level 0 by coarsening space only
        for (size_t l = 1; l < lv.size() && lv[l - 1].to_next == 0; ++l)
            CKS(alloc((void**)&lv[l].x2blk, 32LL * lv[l].g.net * lv[l].g.sp_elems * sizeof(float)));
    }
    storage_tc = tc;
    ws_version++;
    return ST_OK;
}

// 2 x 2 time element matrices of level l ([a_t][b_t], row-major): level 0's upwind
// D_t = [[0, 0], [-1, 1]] and M_t = dt/6 [[2, 1], [1, 2]], then, for every coarsening that halves
// time, the Galerkin product over the two fine slabs of a coarse slab with the nested linear
// interpolation (fine nodes: c0, (c0 + c1) / 2, c1).
static void level_time_mats(const Mesh* m, int l, double Dt[4], double Mt[4]) {
    const double dt = m->lv[0].g.dt;
    double D[4] = {0.0, 0.0, -1.0, 1.0}, Mm[4] = {dt / 3.0, dt / 6.0, dt / 6.0, dt / 3.0};
    auto coarsen = [](double* T) {
        const double P1[2][2] = {{1.0, 0.0}, {0.5, 0.5}}, P2[2][2] = {{0.5, 0.5}, {0.0, 1.0}};
        double C[4] = {0.0, 0.0, 0.0, 0.0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j)
                        C[a * 2 + b] += P1[i][a] * T[i * 2 + j] * P1[j][b] + P2[i][a] * T[i * 2 + j] * P2[j][b];
        for (int q = 0; q < 4; ++q) T[q] = C[q];
    };
    for (int q = 0; q < l; ++q)
        if (m->lv[q].to_next == 1 || m->lv[q].to_next == 2) {
            coarsen(D);
            coarsen(Mm);
        }
    for (int q = 0; q < 4; ++q) {
        Dt[q] = D[q];
        Mt[q] = Mm[q];
    }
}

st_status set_design(Mesh* m, const double* gamma, int layout, size_t count, int mem) {
    if (!gamma) return fail(ST_ERR_ARG, "null design");
    if (layout != ST_DESIGN_EXTRUDED && layout != ST_DESIGN_SPACETIME) return fail(ST_ERR_ARG, "unknown layout");
    const Geom& g0 = m->lv[0].g;
    const long long want = layout == ST_DESIGN_EXTRUDED ? g0.sp_elems : g0.sp_elems * g0.net;
    if ((long long)count != want)
        return fail(ST_ERR_ARG, "design count " + std::to_string(count) + " != " + std::to_string(want));
    cudaSetDevice(m->device);
    if (m->design_count != want) {
        m->drop_graphs();
        m->release(m->g64);
        m->release(m->g16);
        m->release(m->gin);
        m->release(m->gsens);
        m->g64 = nullptr;
        m->g16 = nullptr;
        // padding: the marching kernels copy whole 16-byte chunks of the designs
        CKS(m->alloc((void**)&m->g64, (want + 8) * sizeof(double)));
        CKS(m->alloc((void**)&m->g16, (want + 8) * sizeof(__nv_bfloat16)));
        CKS(m->alloc((void**)&m->gin, want * sizeof(double)));
        CKS(m->alloc((void**)&m->gsens, want * sizeof(double)));
        m->design_count = want;
        m->ws_version++;
    }
    m->layout = layout;
    CKS(m->ensure_level_storage());
    cudaStream_t s = m->stream;
    CK(cudaMemcpyAsync(m->gin, gamma, want * sizeof(double),
                       mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(m->d_err + 2, 0, sizeof(int), s));
    launch_design_cast(m->gin, m->g64, m->g16, want, m->d_err + 2, s);
    // Galerkin coarse operators, level by level, in FP64; FP32 copies for the mixed V-cycle.
    const int L = (int)m->lv.size();
    for (int l = 1; l < L; ++l) {
        const int kind = m->lv[l - 1].to_next;
        if (l == 1)
            launch_build_from_l0(m->sd, m->op0<double>(), m->lv[1].g, kind, m->storage_tc, m->lv[1].e64, s);
        else
            launch_build_from_lc(m->sd, m->opc<double>(l - 1), m->lv[l].g, kind, m->lv[l].e64, s);
        launch_to_float(m->lv[l].e64, m->lv[l].e32, m->lv[l].nstore * nvals(m->sd), s);
    }
    // the two stencils of every coarse level of extruded 3-D designs (FP32 marching kernels)
    for (int l = 1; l < L; ++l) {
        if (!m->lv[l].x3st) continue;
        double Dt[4], Mt[4];
        level_time_mats(m, l, Dt, Mt);
        launch_x3_stencil(m->opc<double>(l), Dt, Mt, m->lv[l].x3st, s);
        for (int q = 0; q < 4; ++q) {
            m->lv[l].x3tw[q] = (float)Dt[q];
            m->lv[l].x3tw[4 + q] = (float)Mt[q];
        }
    }
    // M and K rows of the space-coarsened levels of space-time 2-D designs
    for (int l = 1; l < L; ++l)
        if (m->lv[l].x2blk) launch_x2_blocks(m->opc<double>(l), m->lv[l].x2blk, s);
    // 27-point stencils of every level (extruded designs, 2 spatial dimensions)
    if (m->lv[0].sdir) {
        for (int l = 0; l < L; ++l) {
            OpL0<double> o0 = m->op0<double>();
            OpLc<double> oc = m->opc<double>(l);
            launch_stencil_build(l, o0, oc, m->lv[l].st64, m->lv[l].st32, m->lv[l].sdir, s);
        }
    }
    // coarsest operator, dense, and its inverse (the iterative coarsest solve needs only its
    // Jacobi diagonal, built with the multigrid workspace)
    int herr = 0, htmo = 0;
    if (!m->coarse_iter) {
        const int nc = (int)m->lv[L - 1].g.nnodes;
        launch_dense_assemble(m->sd, L - 1, m->op0<double>(), m->opc<double>(L - 1), m->Ainv, s);
        CK(cudaMemsetAsync(m->d_err, 0, sizeof(int), s));
        CK(cudaMemsetAsync(m->d_err + 3, 0, sizeof(int), s));
        launch_gauss_jordan(m->Ainv, m->Awork, m->pinv, m->gjpr, nc, m->d_err, m->d_bar, m->d_err + 3, s);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&herr, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&htmo, m->d_err + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    int gbad = 0;
    CK(cudaMemcpyAsync(&gbad, m->d_err + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    m->design_version++;
    if (htmo) {
        m->have_design = false;
        m->have_state = false;
        m->have_adjoint = false;
        return fail(ST_ERR_TIMEOUT, "a grid barrier of the coarsest-level inverse gave up waiting");
    }
    if (gbad || herr) {
        // the operators now hold a rejected design: no solve until a valid one is set
        m->have_design = false;
        m->have_state = false;
        m->have_adjoint = false;
        return fail(ST_ERR_NUMERIC, gbad ? "the design holds a NaN or infinite value"
                                         : "zero pivot in the coarsest-level inverse");
    }
    m->have_design = true;
    m->have_state = false;
    m->have_adjoint = false;
    return ST_OK;
}

// ---------------------------------------------------------------- multigrid workspace
template <typename T>
MGWork<T>& Mesh::work() {
    if constexpr (sizeof(T) == 4)
        return w32;
    else
        return w64;
}

template <typename T>
st_status Mesh::ensure_mg(int steps) {
    MGWork<T>& W = work<T>();
    const int L = (int)lv.size();
    if (!W.ready) {
        W.b.assign(L, nullptr);
        W.x.assign(L, nullptr);
        W.r.assign(L, nullptr);
        W.w.assign(L, nullptr);
        W.w2.assign(L, nullptr);
        W.dinv.assign(L, nullptr);
        W.U.assign(L, Basis<T>{});
        for (int l = 0; l < L; ++l) {
            const long long N = lv[l].g.nnodes;
            CKS(alloc((void**)&W.b[l], N * sizeof(T)));
            CKS(alloc((void**)&W.x[l], N * sizeof(T)));
            CKS(alloc((void**)&W.r[l], N * sizeof(T)));
            CKS(alloc((void**)&W.dinv[l], N * sizeof(T)));
            if (l < L - 1) {
                CKS(alloc((void**)&W.w[l], N * sizeof(T)));
                CKS(alloc((void**)&W.w2[l], N * sizeof(T)));
            }
        }
        W.nbasis = 0;
        W.ready = true;
        W.dinv_version = -1;
    }
    if (desc.smoother == ST_SMOOTH_GMRES && steps + 1 > W.nbasis) {  // Jacobi sweeps keep no Krylov basis
        drop_graphs();
        ws_version++;
        for (int l = 0; l < L - 1; ++l) {
            const long long N = lv[l].g.nnodes;
            for (int q = W.nbasis; q <= steps; ++q) CKS(alloc((void**)&W.U[l].u[q], N * sizeof(T)));
        }
        W.nbasis = steps + 1;
    }
    if (coarse_iter && cg_dinv_version != design_version) {
        if (L == 1)
            launch_diag_l0<double>(sd, op0<double>(), cg_dinv, true, stream);
        else
            launch_diag_lc<double>(sd, opc<double>(L - 1), cg_dinv, true, stream);
        cg_dinv_version = design_version;
    }
    if (W.dinv_version != design_version) {
        for (int l = 0; l < L; ++l) {
            if (l == 0)
                launch_diag_l0<T>(sd, op0<T>(), W.dinv[0], true, stream);
            else
                launch_diag_lc<T>(sd, opc<T>(l), W.dinv[l], true, stream);
        }
        // stencil levels that smooth: interior stencils scaled by the Jacobi diagonal
        W.sc.resize(L, nullptr);
        for (int l = 0; l + 1 < L; ++l) {
            if (!lv[l].sdir) continue;
            const long long P = (long long)lv[l].g.nx1 * lv[l].g.ny1;
            if (!W.sc[l]) CKS(alloc((void**)&W.sc[l], 2 * 27 * P * sizeof(T)));
            const T* stl = std::is_same<T, float>::value ? (const T*)lv[l].st32 : (const T*)lv[l].st64;
            launch_stencil_scale<T>(lv[l].g, stl, W.dinv[l], lv[l].sdir, W.sc[l], stream);
        }
        W.dinv_version = design_version;
    }
    if (vt_first >= 0 && (W.vt_version != ws_version || W.steps_uploaded != steps)) CKS(upload_vtail<T>(steps));
    return ST_OK;
}

template <typename T>
st_status Mesh::upload_vtail(int steps) {
    MGWork<T>& W = work<T>();
    if (!W.d_vt) CKS(alloc((void**)&W.d_vt, sizeof(VTail<T>)));
    VTail<T>* h = new VTail<T>();
    memset(h, 0, sizeof(VTail<T>));
    h->first = vt_first;
    h->L = (int)lv.size();
    h->steps = steps;
    h->nc = (int)lv.back().g.nnodes;
    h->Ainv = Ainv;
    h->part = vt_part;
    h->bar = d_bar;
    h->err = d_err + 1;
    h->spin_limit = vt_spin_limit;
    if (vt_trace) {
        h->trace = vt_trace;
        h->trace_cap = 4096;
    }
    h->op0 = op0<T>();
    for (int l = 0; l < (int)lv.size(); ++l) {
        VLevel<T>& V = h->lv[l];
        V.g = lv[l].g;
        V.lv = l;
        V.to_next = lv[l].to_next;
        V.tc = layout == ST_DESIGN_EXTRUDED ? 1 : 0;
        if (l == 0) {
            const OpL0<T> o = op0<T>();
            V.coef[0] = o.st_coef[0];
            V.coef[1] = o.st_coef[1];
            V.dir = o.st_dir;
        } else {
            const OpLc<T> o = opc<T>(l);
            V.coef[0] = o.st_coef[0];
            V.coef[1] = o.st_coef[1];
            V.dir = o.st_dir;
            V.elem = o.elem;
        }
        V.b = W.b[l];
        V.x = W.x[l];
        V.r = W.r[l];
        V.w = W.w[l];
        V.dinv = W.dinv[l];
        for (int q = 0; q <= kMaxSmooth; ++q) V.U[q] = W.U[l].u[q];
    }
    W.steps_uploaded = steps;
    cudaError_t e = cudaMemcpy(W.d_vt, h, sizeof(VTail<T>), cudaMemcpyHostToDevice);
    delete h;
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, std::string("vtail upload: ") + cudaGetErrorString(e));
    W.vt_version = ws_version;
    return ST_OK;
}

// Coarsest level solved by FP64 right-Jacobi-preconditioned restarted GMRES(cg_m) to the
// relative tolerance coarse_rtol (the paper's coarsest solve, Sec. 3.2): the smoother's
// kernels, restarted cg_cycles times, with a stop test in its device state so that the
// fixed launch sequence (graph capturable) does no work after convergence.
template <typename T>
void Mesh::coarse_gmres(bool tr) {
    MGWork<T>& W = work<T>();
    const int l = (int)lv.size() - 1;
    const long long n = lv[l].g.nnodes;
    if constexpr (std::is_same<T, double>::value)
        cudaMemcpyAsync(cg_b, W.b[l], n * sizeof(double), cudaMemcpyDeviceToDevice, stream);
    else
        launch_convert<float, double>(W.b[l], cg_b, n, stream);
    launch_cg_begin<double>(d_smc, desc.coarse_rtol > 0 ? desc.coarse_rtol : 1e-6, stream);
    for (int c = 0; c < cg_cycles; ++c)
        launch_smooth<double>(sd, l, op0<double>(), opc<double>(l), tr, cg_b, cg_x, cg_dinv, cg_U, cg_w, cg_w2, cg_m,
                              c == 0, d_smc, rb, stream, nullptr);
    if constexpr (std::is_same<T, double>::value)
        cudaMemcpyAsync(W.x[l], cg_x, n * sizeof(double), cudaMemcpyDeviceToDevice, stream);
    else
        launch_convert<double, float>(cg_x, W.x[l], n, stream);
}

template <typename T>
void Mesh::smooth(int l, bool tr, bool zero_init, int steps) {
    MGWork<T>& W = work<T>();
    if (desc.smoother == ST_SMOOTH_JACOBI) {  // the residual vector of the level is free during smoothing
        launch_jacobi_smooth<T>(sd, l, op0<T>(), opc<T>(l), tr, W.b[l], W.x[l], W.dinv[l], W.r[l], steps, zero_init,
                                (T)desc.smoother_omega, stream);
        return;
    }
    cudaEvent_t* ev = nullptr;
    if (at_on && l == 0 && l < (int)lv.size() - 1) {
        ev = at_ev + (zero_init ? 0 : 2 * kMaxSmooth);
        at_steps = steps;
    }
    const T* sc = (l < (int)W.sc.size() && lv[l].sdir) ? W.sc[l] : nullptr;
    launch_smooth<T>(sd, l, op0<T>(), opc<T>(l), tr, W.b[l], W.x[l], W.dinv[l], W.U[l], W.w[l], W.w2[l], steps,
                     zero_init, d_sm, rb, stream, ev, sc);
}

// One V-cycle on level l: pre-smoothing from zero, residual, restriction, coarse
// correction, prolongation, post-smoothing (classical V-cycle, Sec. 3.2).
template <typename T>
void Mesh::vcycle_rec(int l, bool tr, int steps) {
    MGWork<T>& W = work<T>();
    const int L = (int)lv.size();
    if (l == L - 1) {
        if (coarse_iter)
            coarse_gmres<T>(tr);
        else
            launch_coarse_solve<T>(Ainv, (int)lv[l].g.nnodes, tr, W.b[l], W.x[l], stream);
        return;
    }
    const bool timing = level_timing && !capturing;
    auto mark = [&](int k) {
        if (timing) cudaEventRecord(tev[l * 4 + k], stream);
    };
    const bool vt_ok = desc.smoother == ST_SMOOTH_GMRES;  // the persistent tail smooths with GMRES only
    if (vt_ok && l == vt_first && W.d_vt && W.steps_uploaded == steps && !vt_failed) {
        mark(0);
        if (launch_vtail<T>(sd, tr, W.d_vt, d_bar, stream) < 0) {
            // the cooperative launch was refused (for example not all blocks can be resident in
            // this context): clear the error and run these levels one launch per phase below
            cudaGetLastError();
            vt_failed = true;
            if (getenv("ST_VERBOSE")) fprintf(stderr, "st: persistent coarse tail refused; one launch per phase\n");
        }
    }
    if (vt_ok && l == vt_first && W.d_vt && W.steps_uploaded == steps && !vt_failed) {
        if (timing) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            cudaEventRecord(e, stream);
            cudaEventSynchronize(e);
            float a = 0;
            cudaEventElapsedTime(&a, tev[l * 4 + 0], e);
            tacc[l * 3] += a;
            cudaEventDestroy(e);
        }
        return;
    }
    mark(0);
    smooth<T>(l, tr, true, steps);
    mark(1);
    launch_residual<T>(sd, l, op0<T>(), opc<T>(l), tr, W.b[l], W.x[l], W.r[l], stream);
    launch_restrict<T>(lv[l].g, lv[l + 1].g, lv[l].to_next, sd, W.r[l], W.b[l + 1], stream);
    mark(2);
    vcycle_rec<T>(l + 1, tr, steps);
    if (timing) cudaEventRecord(tev[l * 4 + 3], stream);
    launch_prolong<T>(lv[l].g, lv[l + 1].g, lv[l].to_next, sd, W.x[l + 1], W.x[l], stream);
    smooth<T>(l, tr, false, steps);
    if (timing) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, stream);
        cudaEventSynchronize(e);
        float a = 0, b = 0, c = 0;
        cudaEventElapsedTime(&a, tev[l * 4 + 0], tev[l * 4 + 1]);
        cudaEventElapsedTime(&b, tev[l * 4 + 1], tev[l * 4 + 2]);
        cudaEventElapsedTime(&c, tev[l * 4 + 3], e);
        tacc[l * 3] += a;
        tacc[l * 3 + 1] += b;
        tacc[l * 3 + 2] += c;
        cudaEventDestroy(e);
        if (l == 0) ++tcycles;
    }
}

template <typename T>
st_status Mesh::vcycle(bool tr, int steps, bool graphs) {
    const int slot = (sizeof(T) == 4 ? 0 : 2) + (tr ? 1 : 0);
    if (at_on && lv.size() > 1) at_pending = true;
    if (!graphs) {
        vcycle_rec<T>(0, tr, steps);
        return ST_OK;
    }
    if (!gexec[slot] || gsteps[slot] != steps) {
        if (gexec[slot]) cudaGraphExecDestroy(gexec[slot]);
        gexec[slot] = nullptr;
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        vcycle_rec<T>(0, tr, steps);
        capturing = false;
        CK(cudaStreamEndCapture(stream, &graph));
        long long graph_kernel_count = 0;
        {
            size_t nn = 0;
            cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
            for (size_t q = 0; q < nn; ++q) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                    ++graph_kernel_count;
            }
        }
        cudaError_t e = cudaGraphInstantiate(&gexec[slot], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gexec[slot] = nullptr;
            return fail(ST_ERR_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
        }
        gsteps[slot] = steps;
        gversion[slot] = design_version;
        gkernels[slot] = graph_kernel_count;
    }
    CK(cudaGraphLaunch(gexec[slot], stream));
    note_graph_launch(gkernels[slot]);
    return ST_OK;
}

// ---------------------------------------------------------------- FGMRES (FP64, right preconditioned)
template <typename T>
st_status Mesh::ensure_krylov(int m, int steps) {
    CKS(ensure_mg<T>(steps));
    std::vector<T*>& Z = sizeof(T) == 4 ? (std::vector<T*>&)Z32 : (std::vector<T*>&)Z64;
    const long long N = lv[0].g.nnodes;
    while ((int)V.size() < m + 1) {
        double* p = nullptr;
        CKS(alloc((void**)&p, N * sizeof(double)));
        V.push_back(p);
    }
    while ((int)Z.size() < m) {
        T* p = nullptr;
        CKS(alloc((void**)&p, N * sizeof(T)));
        Z.push_back(p);
    }
    return ST_OK;
}

template <typename T>
st_status Mesh::fgmres(bool tr, const double* rhs, double* x, const st_options& o, st_stats* stats) {
    const Geom& g = lv[0].g;
    const int m = o.restart;
    CKS(ensure_krylov<T>(m, o.smooth_steps));
    MGWork<T>& W = work<T>();
    std::vector<T*>& Z = sizeof(T) == 4 ? (std::vector<T*>&)Z32 : (std::vector<T*>&)Z64;
    const long long N = g.nnodes;
    const OpL0<double> A64 = op0<double>();
    cudaStream_t s = stream;
    // ||f||
    launch_dot64(g, rhs, rhs, d_scalar, rb, s);
    double nf2 = 0;
    CK(cudaMemcpyAsync(&nf2, d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double nf = sqrt(nf2);
    stats->norm_f = nf;
    stats->outer_its = 0;
    stats->restarts = 0;
    stats->converged = 0;
    if (!std::isfinite(nf)) return fail(ST_ERR_NUMERIC, "NaN/Inf in the right-hand side");
    if (!(nf > 0)) {
        CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        CK(cudaStreamSynchronize(s));
        stats->converged = 1;
        stats->rel_res = 0;
        stats->rel_res_est = 0;
        return ST_OK;
    }
    const double tol = o.rtol * nf;
    int its = 0;
    auto read_fg = [&]() -> st_status {
        CK(cudaMemcpyAsync(h_fg, d_fg, sizeof(FgState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        timer_collect();
        return ST_OK;
    };
    launch_fg_residual(sd, A64, tr, rhs, x, V[0], d_fg, rb, s);
    CKS(read_fg());
    double beta = h_fg->beta;
    st_status result = ST_OK;
    for (;;) {
        if (!(beta == beta) || h_fg->bad) {
            result = fail(ST_ERR_NUMERIC, "NaN/Inf in the residual");
            break;
        }
        if (beta <= tol) {
            stats->converged = 1;
            break;
        }
        if (its >= o.max_it) {
            result = fail(ST_ERR_NOT_CONVERGED, "rtol not reached within max_it outer iterations");
            break;
        }
        launch_fg_start<T>(g, V[0], W.b[0], d_fg, s);
        int k = 0;
        for (int j = 0; j < m; ++j) {
            CKS(vcycle<T>(tr, o.smooth_steps, o.use_graphs != 0));
            launch_fg_apply_dots<T>(sd, A64, tr, W.x[0], Z[j], fg_w, V.data(), j, d_fg, rb, s);
            launch_fg_update_dots(g, fg_w, V.data(), j, 0, d_fg, rb, s);
            launch_fg_update_dots(g, fg_w, V.data(), j, 1, d_fg, rb, s);
            ++its;
            k = j + 1;
            CKS(read_fg());
            if (h_fg->bad) break;
            if (h_fg->res_est <= tol || h_fg->breakdown || its >= o.max_it) break;
            launch_fg_normalize<T>(g, fg_w, V[j + 1], W.b[0], j, d_fg, s);
        }
        stats->rel_res_est = h_fg->res_est / nf;
        if (h_fg->bad) {
            result = fail(ST_ERR_NUMERIC, "NaN/Inf in the Arnoldi process");
            break;
        }
        launch_fg_update_x<T>(g, x, Z.data(), k, d_fg, s);
        launch_fg_residual(sd, A64, tr, rhs, x, V[0], d_fg, rb, s);
        CKS(read_fg());
        beta = h_fg->beta;
        stats->restarts++;
    }
    if (stats->restarts > 0) stats->restarts--;
    stats->outer_its = its;
    stats->rel_res = beta / nf;
    CK(cudaGetLastError());
    return result;
}

// ---------------------------------------------------------------- graph-resident restart cycles
// Adds a conditional node (WHILE or SWITCH with `size` bodies) at the current end of the
// capture on stream s and makes it the new end; returns the body graphs.
static st_status add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                 unsigned size, cudaGraph_t** bodies) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &nd));
    if (cst != cudaStreamCaptureStatusActive) return fail(ST_ERR_CUDA, "conditional node outside a capture");
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *bodies = p.conditional.phGraph_out;
    return ST_OK;
}

template <typename T>
st_status Mesh::capture_cycle(cudaGraph_t G, cudaStream_t* cs, bool tr, const st_options& o, double tol,
                              const double* rhs, double* x, long long* per_iter, long long* fixed) {
    const Geom& g = lv[0].g;
    const int m = o.restart;
    MGWork<T>& W = work<T>();
    std::vector<T*>& Z = sizeof(T) == 4 ? (std::vector<T*>&)Z32 : (std::vector<T*>&)Z64;
    const OpL0<double> A64 = op0<double>();
    cudaGraphConditionalHandle hw, hs;
    CK(cudaGraphConditionalHandleCreate(&hw, G, 0, cudaGraphCondAssignDefault));
    cudaStream_t keep = stream;
    const bool keep_pdl = g_no_pdl;
    g_no_pdl = true;
    // conditional bodies hold kernels, memory copies and conditionals only: no timing events
    // and no cooperative tail launch inside them
    const bool keep_at = at_on;
    const int keep_vt = vt_first;
    at_on = false;
    vt_first = -1;
    st_status r = ST_OK;
    long long vk = 0;
    auto body = [&]() -> st_status {
        CK(cudaStreamBeginCaptureToGraph(cs[0], G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        launch_fg_residual(sd, A64, tr, rhs, x, V[0], d_fg, rb, cs[0]);
        launch_fg_begin(d_fg, tol, o.max_it, hw, cs[0]);
        launch_fg_start<T>(g, V[0], W.b[0], d_fg, cs[0]);
        cudaGraph_t* wb = nullptr;
        CKS(add_conditional(cs[0], hw, cudaGraphCondTypeWhile, 1, &wb));
        // WHILE body: the iteration index for the SWITCH, the V-cycle, the iteration's kernels, loop test
        CK(cudaGraphConditionalHandleCreate(&hs, wb[0], 0, 0));
        CK(cudaStreamBeginCaptureToGraph(cs[1], wb[0], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        launch_fg_setj(d_fg, hs, cs[1]);
        stream = cs[1];
        vcycle_rec<T>(0, tr, o.smooth_steps);
        stream = keep;
        {
            size_t nn = 0;
            cudaGraph_t cg = nullptr;
            cudaStreamCaptureStatus cst;
            CK(cudaStreamGetCaptureInfo(cs[1], &cst, nullptr, &cg, nullptr, nullptr, nullptr));
            CK(cudaGraphGetNodes(cg, nullptr, &nn));
            vk = (long long)nn;  // the V-cycle's kernels and the index kernel
        }
        cudaGraph_t* sb = nullptr;
        CKS(add_conditional(cs[1], hs, cudaGraphCondTypeSwitch, (unsigned)m, &sb));
        for (int j = 0; j < m; ++j) {
            CK(cudaStreamBeginCaptureToGraph(cs[2], sb[j], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            launch_fg_apply_dots<T>(sd, A64, tr, W.x[0], Z[j], fg_w, V.data(), j, d_fg, rb, cs[2]);
            launch_fg_update_dots(g, fg_w, V.data(), j, 0, d_fg, rb, cs[2]);
            launch_fg_update_dots(g, fg_w, V.data(), j, 1, d_fg, rb, cs[2]);
            launch_fg_check(d_fg, j, tol, o.max_it, m, cs[2]);
            if (j + 1 < m) launch_fg_normalize<T>(g, fg_w, V[j + 1], W.b[0], j, d_fg, cs[2]);
            cudaGraph_t tmp;
            CK(cudaStreamEndCapture(cs[2], &tmp));
        }
        launch_fg_loop(d_fg, hw, cs[1]);
        cudaGraph_t tmp;
        CK(cudaStreamEndCapture(cs[1], &tmp));
        launch_fg_update_x_dev<T>(g, x, Z.data(), m, d_fg, cs[0]);
        launch_fg_residual(sd, A64, tr, rhs, x, V[0], d_fg, rb, cs[0]);
        CK(cudaStreamEndCapture(cs[0], &tmp));
        return ST_OK;
    };
    r = body();
    capturing = false;
    stream = keep;
    g_no_pdl = keep_pdl;
    at_on = keep_at;
    vt_first = keep_vt;
    if (r != ST_OK) {
        // end any capture left open by the failure
        for (int q = 2; q >= 0; --q) {
            cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(cs[q], &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(cs[q], &tmp);
            }
        }
        cudaGetLastError();
        return r;
    }
    *per_iter = vk + 7;  // V-cycle and index kernel, apply + 3 passes, check, normalize, loop test
    *fixed = 7;          // residual, begin, start, back substitution, combination, residual
    return ST_OK;
}

st_status solve(Mesh* m, bool adjoint, const st_options* op, st_stats* stats) {
    st_options o;
    st_options_default(&o);
    if (op) o = *op;
    if (o.restart < 1 || o.restart > kMaxRestart) return fail(ST_ERR_ARG, "restart must be in [1, 32]");
    if (o.smooth_steps < 1 || o.smooth_steps > kMaxSmooth) return fail(ST_ERR_ARG, "smooth_steps must be in [1, 16]");
    if (!(o.rtol > 0) || o.max_it < 1) return fail(ST_ERR_ARG, "rtol and max_it must be positive");
    if (o.precision != ST_PREC_MIXED && o.precision != ST_PREC_FP64) return fail(ST_ERR_ARG, "unknown precision");
    st_stats local{};
    st_stats* S = stats ? stats : &local;
    *S = st_stats{};
    const double t0 = now_s();
    double* x = adjoint ? m->lam : m->s;
    const double* rhs = adjoint ? m->adjrhs : m->f;
    if (!o.warm_start) CK(cudaMemsetAsync(x, 0, m->lv[0].g.nnodes * sizeof(double), m->stream));
    CK(cudaMemsetAsync(m->d_err + 1, 0, sizeof(int), m->stream));
    st_status r = o.precision == ST_PREC_MIXED ? m->fgmres<float>(adjoint, rhs, x, o, S)
                                               : m->fgmres<double>(adjoint, rhs, x, o, S);
    cudaStreamSynchronize(m->stream);
    int tmo = 0;
    cudaMemcpy(&tmo, m->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (tmo) r = fail(ST_ERR_TIMEOUT, "a grid barrier of the coarse V-cycle tail gave up waiting");
    S->seconds = now_s() - t0;
    return r;
}

st_status solve_batch(Mesh* const* ms, int n, bool adjoint, const st_options* op, st_stats* stats,
                      st_status* status) {
    st_options o;
    st_options_default(&o);
    if (op) o = *op;
    if (n < 1 || !ms) return fail(ST_ERR_ARG, "empty batch");
    if (o.restart < 1 || o.restart > kMaxRestart) return fail(ST_ERR_ARG, "restart must be in [1, 32]");
    if (o.smooth_steps < 1 || o.smooth_steps > kMaxSmooth) return fail(ST_ERR_ARG, "smooth_steps must be in [1, 16]");
    if (!(o.rtol > 0) || o.max_it < 1) return fail(ST_ERR_ARG, "rtol and max_it must be positive");
    if (o.precision != ST_PREC_MIXED && o.precision != ST_PREC_FP64) return fail(ST_ERR_ARG, "unknown precision");
    for (int k = 0; k < n; ++k) {
        if (!ms[k]) return fail(ST_ERR_ARG, "null mesh in the batch");
        if (ms[k]->device != ms[0]->device) return fail(ST_ERR_ARG, "the meshes of a batch must share a device");
        for (int q = 0; q < k; ++q)
            if (ms[q] == ms[k]) return fail(ST_ERR_ARG, "a mesh appears twice in the batch");
    }
    const bool mixed = o.precision == ST_PREC_MIXED;
    const double t0 = now_s();
    cudaSetDevice(ms[0]->device);
    std::vector<st_stats> S(n);
    std::vector<st_status> R(n, ST_OK);
    std::vector<double> nf(n, 0.0), tol(n, 0.0);
    std::vector<char> active(n, 0);
    // storage, initial guess, ||f|| (one synchronisation per mesh stream)
    for (int k = 0; k < n; ++k) {
        Mesh* m = ms[k];
        CKS(mixed ? m->ensure_krylov<float>(o.restart, o.smooth_steps) : m->ensure_krylov<double>(o.restart, o.smooth_steps));
        double* x = adjoint ? m->lam : m->s;
        const double* rhs = adjoint ? m->adjrhs : m->f;
        if (!o.warm_start) CK(cudaMemsetAsync(x, 0, m->lv[0].g.nnodes * sizeof(double), m->stream));
        CK(cudaMemsetAsync(&m->d_fg->its, 0, sizeof(int), m->stream));
        launch_dot64(m->lv[0].g, rhs, rhs, m->d_scalar, m->rb, m->stream);
        CK(cudaMemcpyAsync(&nf[k], m->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    }
    for (int k = 0; k < n; ++k) CK(cudaStreamSynchronize(ms[k]->stream));
    int n_active = 0;
    for (int k = 0; k < n; ++k) {
        nf[k] = sqrt(nf[k]);
        S[k].norm_f = nf[k];
        if (!std::isfinite(nf[k])) {
            R[k] = fail(ST_ERR_NUMERIC, "NaN/Inf in the right-hand side");
        } else if (!(nf[k] > 0)) {
            double* x = adjoint ? ms[k]->lam : ms[k]->s;
            CK(cudaMemsetAsync(x, 0, ms[k]->lv[0].g.nnodes * sizeof(double), ms[k]->stream));
            CK(cudaStreamSynchronize(ms[k]->stream));
            S[k].converged = 1;
        } else {
            tol[k] = o.rtol * nf[k];
            active[k] = 1;
            ++n_active;
        }
    }
    if (n_active > 0) {
        cudaStream_t bs = ms[0]->stream;
        cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
        cudaGraph_t G = nullptr;
        cudaGraphExec_t X = nullptr;
        std::vector<long long> per_iter(n, 0), fixed(n, 0);
        std::vector<int> its_prev(n, 0), cycles(n, 0);
        st_status r = ST_OK;
        auto run = [&]() -> st_status {
            for (int q = 0; q < 3; ++q) CK(cudaStreamCreateWithFlags(&cs[q], cudaStreamNonBlocking));
            CK(cudaGraphCreate(&G, 0));
            for (int k = 0; k < n; ++k) {
                if (!active[k]) continue;
                Mesh* m = ms[k];
                double* x = adjoint ? m->lam : m->s;
                const double* rhs = adjoint ? m->adjrhs : m->f;
                if (mixed)
                    CKS(m->capture_cycle<float>(G, cs, adjoint, o, tol[k], rhs, x, &per_iter[k], &fixed[k]));
                else
                    CKS(m->capture_cycle<double>(G, cs, adjoint, o, tol[k], rhs, x, &per_iter[k], &fixed[k]));
            }
            const cudaError_t e = cudaGraphInstantiate(&X, G, 0);
            if (e != cudaSuccess) {
                X = nullptr;
                return fail(ST_ERR_CUDA, std::string("batch graph instantiation failed: ") + cudaGetErrorString(e));
            }
            // one launch advances every unfinished mesh by a restart cycle; finished meshes only
            // recompute their residual
            for (int launch = 0; launch <= o.max_it + 1; ++launch) {
                CK(cudaGraphLaunch(X, bs));
                for (int k = 0; k < n; ++k)
                    if (active[k]) CK(cudaMemcpyAsync(ms[k]->h_fg, ms[k]->d_fg, sizeof(FgState), cudaMemcpyDeviceToHost, bs));
                CK(cudaStreamSynchronize(bs));
                bool more = false;
                long long kernels = 0;
                for (int k = 0; k < n; ++k) {
                    if (!active[k]) continue;
                    const FgState* f = ms[k]->h_fg;
                    kernels += fixed[k] + per_iter[k] * (f->its - its_prev[k]);
                    if (f->its > its_prev[k]) ++cycles[k];
                    its_prev[k] = f->its;
                    const double beta = f->beta;
                    S[k].outer_its = f->its;
                    S[k].rel_res = beta / nf[k];
                    S[k].rel_res_est = f->res_est / nf[k];
                    if (!(beta == beta) || f->bad) {
                        R[k] = fail(ST_ERR_NUMERIC, "NaN/Inf in the residual or the Arnoldi process");
                    } else if (beta <= tol[k]) {
                        S[k].converged = 1;
                        R[k] = ST_OK;
                    } else if (f->its >= o.max_it) {
                        R[k] = fail(ST_ERR_NOT_CONVERGED, "rtol not reached within max_it outer iterations");
                    } else {
                        more = true;
                    }
                }
                note_graph_launch(kernels);
                if (!more) break;
            }
            return ST_OK;
        };
        r = run();
        if (X) cudaGraphExecDestroy(X);
        if (G) cudaGraphDestroy(G);
        for (int q = 0; q < 3; ++q)
            if (cs[q]) cudaStreamDestroy(cs[q]);
        if (r != ST_OK) return r;
        for (int k = 0; k < n; ++k) S[k].restarts = cycles[k] > 0 ? cycles[k] - 1 : 0;
    }
    const double t = now_s() - t0;
    st_status worst = ST_OK;
    for (int k = 0; k < n; ++k) {
        S[k].seconds = t;
        if (stats) stats[k] = S[k];
        if (status) status[k] = R[k];
        if (R[k] != ST_OK && (worst == ST_OK || worst == ST_ERR_NOT_CONVERGED)) worst = R[k];
    }
    if (worst != ST_OK) fail(worst, "a solve of the batch did not succeed (see the per-mesh statuses)");
    return worst;
}

// ---------------------------------------------------------------- PDE filter (Sec. 3.3.2)
// Coefficient table of the filter matrix: for each node class (lower boundary, interior, upper
// boundary along each axis; axes ordered t, [z,] y, x with x fastest) the coefficients of its
// 3^(SD+1) neighbours, products of the 1-D mass (h/6 [1 4 1], boundary diagonal h/3) and
// stiffness (1/h [-1 2 -1], boundary diagonal 1/h) entries of each axis.
static void filter_table(int sd, const double* h, double dt, double rx, double rt, std::vector<double>& tab) {
    const int na = sd + 1;  // axes: 0 = x ... sd-1 spatial, sd = t
    int no = 1;
    for (int a = 0; a < na; ++a) no *= 3;
    tab.assign((size_t)no * no, 0.0);
    auto m1 = [](int c, int o, double hh) {
        if (o == 0) return c == 1 ? 2.0 * hh / 3.0 : hh / 3.0;
        if (o < 0) return c == 0 ? 0.0 : hh / 6.0;
        return c == 2 ? 0.0 : hh / 6.0;
    };
    auto k1 = [](int c, int o, double hh) {
        if (o == 0) return c == 1 ? 2.0 / hh : 1.0 / hh;
        if (o < 0) return c == 0 ? 0.0 : -1.0 / hh;
        return c == 2 ? 0.0 : -1.0 / hh;
    };
    const double Dx = rx * rx / 12.0, Dt = rt * rt / 12.0;
    for (int cls = 0; cls < no; ++cls)
        for (int o = 0; o < no; ++o) {
            int c[4], off[4];
            double sz[4];
            int cc = cls, oo = o;
            for (int a = 0; a < na; ++a) {  // x first (fastest) ... t last
                c[a] = cc % 3;
                off[a] = oo % 3 - 1;
                cc /= 3;
                oo /= 3;
                sz[a] = a < sd ? h[a] : dt;
            }
            double mass = 1.0;
            for (int a = 0; a < na; ++a) mass *= m1(c[a], off[a], sz[a]);
            double v = mass;
            for (int a = 0; a < na; ++a) {
                double t = (a < sd ? Dx : Dt) * k1(c[a], off[a], sz[a]);
                for (int b = 0; b < na; ++b)
                    if (b != a) t *= m1(c[b], off[b], sz[b]);
                v += t;
            }
            tab[(size_t)cls * no + o] = v;
        }
}

st_status filter(Mesh* m, const double* in, double* out, size_t count, int mem, double rx, double rt, double rtol,
                 int max_it, int* iters) {
    if (!in || !out) return fail(ST_ERR_ARG, "null argument");
    const Geom& g0 = m->lv[0].g;
    const bool extruded = (long long)count == g0.sp_elems;
    if (!extruded && (long long)count != g0.sp_elems * g0.net)
        return fail(ST_ERR_ARG, "count must be the number of spatial or space-time elements");
    if (!(rtol > 0) || max_it < 1) return fail(ST_ERR_ARG, "rtol and max_it must be positive");
    Geom fg = g0;
    if (extruded) {  // a time-constant field: one slab (its filtered field is time-constant)
        fg.net = 1;
        fg.nt1 = 2;
        fg.dt = m->desc.tau;
        fg.nnodes = 2 * fg.plane;
    }
    double hmin = fg.h[0];
    for (int d = 1; d < m->sd; ++d) hmin = std::min(hmin, fg.h[d]);
    if (!(rx > 0)) rx = 2.4 * hmin;
    if (!(rt > 0)) rt = 2.4 * g0.dt;
    const long long N = fg.nnodes;
    const int no = m->sd == 2 ? 27 : 81;
    const long long need = 7 * N + 2 * (long long)count + (long long)no * no + 8;
    cudaSetDevice(m->device);
    if (m->fbuf_len < need) {
        m->release(m->fbuf);
        m->fbuf = nullptr;
        m->fbuf_len = 0;
        CKS(m->alloc((void**)&m->fbuf, need * sizeof(double)));
        m->fbuf_len = need;
    }
    double *b = m->fbuf, *x = b + N, *r = x + N, *z = r + N, *p = z + N, *q = p + N, *dinv = q + N;
    double* ein = dinv + N;
    double* eout = ein + count;
    double* tab = eout + count;
    double* sc = tab + (long long)no * no;
    std::vector<double> htab;
    filter_table(m->sd, fg.h, fg.dt, rx, rt, htab);
    cudaStream_t s = m->stream;
    CK(cudaMemcpyAsync(tab, htab.data(), htab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ein, in, count * sizeof(double),
                       mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    double ve = fg.dt;
    for (int d = 0; d < m->sd; ++d) ve *= fg.h[d];
    launch_filter_rhs(m->sd, fg, ein, ve / (double)(1 << (m->sd + 1)), b, s);
    launch_filter_apply(m->sd, fg, tab, nullptr, nullptr, dinv, s);
    CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    CK(cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(p, 0, N * sizeof(double), s));
    launch_cg_zp(N, 0.0, dinv, r, z, p, s);  // z = D^-1 r, p = z
    double hs[2];
    launch_dot64(fg, r, z, sc, m->rb, s);
    launch_dot64(fg, b, b, sc + 1, m->rb, s);
    CK(cudaMemcpyAsync(hs, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double rz = hs[0];
    const double bn = sqrt(hs[1]);
    if (!std::isfinite(bn)) return fail(ST_ERR_NUMERIC, "NaN/Inf in the field to filter");
    int it = 0;
    bool conv = !(bn > 0);
    while (!conv && it < max_it) {
        launch_filter_apply(m->sd, fg, tab, p, q, nullptr, s);
        launch_dot64(fg, p, q, sc, m->rb, s);
        CK(cudaMemcpyAsync(hs, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!(hs[0] > 0) || !std::isfinite(hs[0])) return fail(ST_ERR_NUMERIC, "filter CG breakdown (p^T A p <= 0)");
        const double alpha = rz / hs[0];
        launch_cg_xr(N, alpha, p, q, x, r, s);
        launch_cg_zp(N, 0.0, dinv, r, z, z, s);  // z = D^-1 r
        launch_dot64(fg, r, r, sc, m->rb, s);
        launch_dot64(fg, r, z, sc + 1, m->rb, s);
        CK(cudaMemcpyAsync(hs, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ++it;
        if (!std::isfinite(hs[0])) return fail(ST_ERR_NUMERIC, "NaN/Inf in the filter solve");
        if (sqrt(hs[0]) <= rtol * bn) {
            conv = true;
            break;
        }
        const double beta = hs[1] / rz;
        rz = hs[1];
        launch_cg_p(N, beta, z, p, s);
    }
    launch_filter_mean(m->sd, fg, x, eout, s);
    CK(cudaMemcpyAsync(out, eout, count * sizeof(double),
                       mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (!conv) return fail(ST_ERR_NOT_CONVERGED, "filter CG did not reach rtol within max_it iterations");
    return ST_OK;
}

}  // namespace st

// ================================================================= C ABI
using st::fail;
using st::Mesh;

struct st_mesh : public st::Mesh {};

static Mesh* M(st_mesh* m) { return static_cast<Mesh*>(m); }

namespace st {
Mesh* mesh_of(st_mesh* m) { return M(m); }
}  // namespace st

static st_status finish_sync(Mesh* mm) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

template <typename T>
static st_status smooth_entry(Mesh* mm, int level, int transpose, const void* b, void* x, int steps, int zero_init) {
    CKS(mm->ensure_mg<T>(steps));
    st::MGWork<T>& W = mm->work<T>();
    const long long N = mm->lv[level].g.nnodes;
    CK(cudaMemcpyAsync(W.b[level], b, N * sizeof(T), cudaMemcpyDeviceToDevice, mm->stream));
    CK(cudaMemcpyAsync(W.x[level], x, N * sizeof(T), cudaMemcpyDeviceToDevice, mm->stream));
    if (level == (int)mm->lv.size() - 1 && W.w[level] == nullptr) {
        CKS(mm->alloc((void**)&W.w[level], N * sizeof(T)));
        CKS(mm->alloc((void**)&W.w2[level], N * sizeof(T)));
    }
    if (W.U[level].u[0] == nullptr)
        for (int q = 0; q < W.nbasis; ++q) CKS(mm->alloc((void**)&W.U[level].u[q], N * sizeof(T)));
    mm->smooth<T>(level, transpose != 0, zero_init != 0, steps);
    CK(cudaMemcpyAsync(x, W.x[level], N * sizeof(T), cudaMemcpyDeviceToDevice, mm->stream));
    return finish_sync(mm);
}

template <typename T>
static st_status vcycle_entry(Mesh* mm, int transpose, const void* b, void* x) {
    st_options o;
    st_options_default(&o);
    CKS(mm->ensure_mg<T>(o.smooth_steps));
    st::MGWork<T>& W = mm->work<T>();
    const long long N = mm->lv[0].g.nnodes;
    CK(cudaMemcpyAsync(W.b[0], b, N * sizeof(T), cudaMemcpyDeviceToDevice, mm->stream));
    CKS(mm->vcycle<T>(transpose != 0, o.smooth_steps, false));
    CK(cudaMemcpyAsync(x, W.x[0], N * sizeof(T), cudaMemcpyDeviceToDevice, mm->stream));
    const st_status r = finish_sync(mm);
    mm->timer_collect();
    return r;
}

// A source description the right-hand side kernel can integrate on this mesh.
static st_status check_source(const st::Mesh* mm, const st_source& q) {
    if (q.kind != ST_SRC_UNIFORM && q.kind != ST_SRC_SIN_T && q.kind != ST_SRC_GAUSSIAN)
        return st::fail(ST_ERR_ARG, "unknown source kind");
    if (!std::isfinite(q.q0) || !std::isfinite(q.a) || !std::isfinite(q.b) || !std::isfinite(q.f))
        return st::fail(ST_ERR_ARG, "source parameters must be finite");
    if (q.kind == ST_SRC_GAUSSIAN && (mm->sd != 2 || !(q.a > 0)))
        return st::fail(ST_ERR_ARG, "the Gaussian source needs two space dimensions and a positive width");
    return ST_OK;
}

extern "C" {

const char* st_version(void) { return "st-gb300 0.1 (sm_103a)"; }

const char* st_last_error(void) {
    return st::g_last_error_static ? st::g_last_error_static : st::g_last_error.c_str();
}

void st_mesh_desc_default(st_mesh_desc* d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->ndim_space = 2;
    d->n[0] = d->n[1] = d->n[2] = 32;
    d->n_t = 32;
    d->ext[0] = d->ext[1] = d->ext[2] = 1.0;
    d->tau = 1.0;
    d->mat.C_ins = 0.5;
    d->mat.C_con = 1.0;
    d->mat.k_ins = 0.03;
    d->mat.k_con = 3.0;
    d->mat.p_c = 2;
    d->mat.p_k = 3;
    d->bc = ST_BC_PATCH_LEFT;
    d->bc_width = 0.1;
    d->lambda_crit = 0.5;
    d->coarse_dof_cap = 2000;
    d->max_levels = 0;
    d->coarsening = ST_COARSEN_SEMI;
    d->device = 0;
    d->smoother = ST_SMOOTH_GMRES;
    d->smoother_omega = 0.5;
}

void st_options_default(st_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->rtol = 1e-8;
    o->max_it = 200;
    o->restart = 30;
    o->precision = ST_PREC_MIXED;
    o->warm_start = 0;
    o->smooth_steps = 10;
    o->use_graphs = 1;
}

st_status st_plan_hierarchy(const st_mesh_desc* d, st_level_info* out, int max_out, int* n_levels) {
    return st::plan_hierarchy(d, out, max_out, n_levels);
}

long long st_kernel_launches(void) { return st::kernel_launches(); }

st_status st_create_mesh(const st_mesh_desc* d, st_mesh** out) {
    Mesh* m = nullptr;
    st_status s = st::create_mesh(d, &m);
    if (out) *out = static_cast<st_mesh*>(m);
    return s;
}

st_status st_destroy_mesh(st_mesh* m) {
    if (!m) return fail(ST_ERR_ARG, "null mesh");
    delete M(m);
    return ST_OK;
}

st_status st_mesh_info_get(const st_mesh* m, st_mesh_info* info) {
    if (!m || !info) return fail(ST_ERR_ARG, "null argument");
    const Mesh* mm = static_cast<const Mesh*>(m);
    info->n_levels = (int)mm->lv.size();
    info->n_nodes = mm->lv[0].g.nnodes;
    info->n_elem = mm->lv[0].g.sp_elems * mm->lv[0].g.net;
    info->device_bytes = mm->bytes_held;
    return ST_OK;
}

st_status st_level_info_get(const st_mesh* m, int level, st_level_info* info) {
    if (!m || !info) return fail(ST_ERR_ARG, "null argument");
    const Mesh* mm = static_cast<const Mesh*>(m);
    if (level < 0 || level >= (int)mm->lv.size()) return fail(ST_ERR_ARG, "level out of range");
    const st::Geom& g = mm->lv[level].g;
    info->n[0] = g.nex;
    info->n[1] = g.ney;
    info->n[2] = mm->sd == 3 ? g.nez : 0;
    info->n_t = g.net;
    info->n_nodes = g.nnodes;
    info->to_next = mm->lv[level].to_next;
    for (int q = 0; q < 3; ++q) info->h[q] = g.h[q];
    info->dt = g.dt;
    return ST_OK;
}

st_status st_set_stream(st_mesh* m, void* stream) {
    if (!m) return fail(ST_ERR_ARG, "null mesh");
    Mesh* mm = M(m);
    cudaStreamSynchronize(mm->stream);
    mm->stream = stream ? (cudaStream_t)stream : mm->own;
    return ST_OK;
}

st_status st_synchronize(st_mesh* m) {
    if (!m) return fail(ST_ERR_ARG, "null mesh");
    cudaError_t e = cudaStreamSynchronize(M(m)->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

st_status st_set_design(st_mesh* m, const double* gamma, int layout, size_t count, int mem) {
    if (!m) return fail(ST_ERR_ARG, "null mesh");
    cudaSetDevice(M(m)->device);
    return st::set_design(M(m), gamma, layout, count, mem);
}

st_status st_solve_forward(st_mesh* m, const st_source* q, const st_options* o, st_stats* stats) {
    if (!m || !q) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    if (!mm->have_design) return fail(ST_ERR_STATE, "st_set_design must precede st_solve_forward");
    CKS(check_source(mm, *q));
    cudaSetDevice(mm->device);
    st::launch_rhs(mm->sd, mm->lv[0].g, q->kind, q->q0, q->a, q->b, q->f, mm->f, mm->stream);
    st_status r = st::solve(mm, false, o, stats);
    mm->have_state = (r == ST_OK || r == ST_ERR_NOT_CONVERGED);
    mm->have_adjoint = false;
    return r;
}

// Objective phi of the stored state and the adjoint right-hand side (d phi / d s)^T.
static st_status adjoint_rhs(Mesh* mm, const st_objective* obj, double* phi_out) {
    if (!mm->have_state) return fail(ST_ERR_STATE, "st_solve_forward must precede st_solve_adjoint");
    cudaSetDevice(mm->device);
    const st::Geom& g = mm->lv[0].g;
    double phi = 0;
    if (obj->kind == ST_OBJ_COMPLIANCE) {
        st::launch_dot64(g, mm->f, mm->s, mm->d_scalar, mm->rb, mm->stream);
        cudaMemcpyAsync(mm->adjrhs, mm->f, g.nnodes * sizeof(double), cudaMemcpyDeviceToDevice, mm->stream);
        cudaMemcpyAsync(&phi, mm->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, mm->stream);
    } else if (obj->kind == ST_OBJ_PNORM) {
        if (obj->P < 1 || obj->P > 64) return fail(ST_ERR_ARG, "p-norm exponent must be in [1, 64]");
        st::launch_pnorm(mm->sd, g, mm->s, obj->P, mm->adjrhs, mm->d_scalar + 1, mm->rb, mm->d_scalar + 2, mm->stream);
        cudaMemcpyAsync(&phi, mm->d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, mm->stream);
    } else {
        return fail(ST_ERR_ARG, "unknown objective kind");
    }
    cudaError_t e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    if (phi_out) *phi_out = phi;
    return ST_OK;
}

st_status st_solve_adjoint(st_mesh* m, const st_objective* obj, const st_options* o, double* phi_out,
                           st_stats* stats) {
    if (!m || !obj) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(adjoint_rhs(mm, obj, phi_out));
    st_status r = st::solve(mm, true, o, stats);
    mm->have_adjoint = (r == ST_OK || r == ST_ERR_NOT_CONVERGED);
    return r;
}

st_status st_filter(st_mesh* m, const double* in, double* out, size_t count, int mem, double r_x, double r_t,
                    double rtol, int max_it, int* iterations) {
    if (!m) return fail(ST_ERR_ARG, "null mesh");
    return st::filter(M(m), in, out, count, mem, r_x, r_t, rtol, max_it, iterations);
}

st_status st_heaviside(st_mesh* m, const double* in, double* out, double* dout, size_t count, int mem, double beta,
                       double eta) {
    if (!m || !in || (!out && !dout)) return fail(ST_ERR_ARG, "null argument");
    if (!(beta > 0) || !(eta > 0 && eta < 1)) return fail(ST_ERR_ARG, "beta > 0 and 0 < eta < 1 required");
    Mesh* mm = M(m);
    cudaSetDevice(mm->device);
    cudaStream_t s = mm->stream;
    const double* din = in;
    double *o1 = out, *o2 = dout;
    double* tmp = nullptr;
    if (mem == ST_MEM_HOST) {
        CKS(mm->alloc((void**)&tmp, 3 * count * sizeof(double)));
        CK(cudaMemcpyAsync(tmp, in, count * sizeof(double), cudaMemcpyHostToDevice, s));
        din = tmp;
        o1 = out ? tmp + count : nullptr;
        o2 = dout ? tmp + 2 * count : nullptr;
    }
    st::launch_heaviside((long long)count, din, o1, o2, beta, eta, s);
    if (mem == ST_MEM_HOST) {
        if (out) CK(cudaMemcpyAsync(out, o1, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (dout) CK(cudaMemcpyAsync(dout, o2, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (tmp) mm->release(tmp);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

st_status st_solve_forward_batch(st_mesh* const* m, int count, const st_source* q, const st_options* o,
                                 st_stats* stats, st_status* status) {
    if (!m || !q || count < 1) return fail(ST_ERR_ARG, "null argument or empty batch");
    std::vector<Mesh*> ms(count);
    for (int k = 0; k < count; ++k) {
        if (!m[k]) return fail(ST_ERR_ARG, "null mesh in the batch");
        ms[k] = M(m[k]);
        if (!ms[k]->have_design) return fail(ST_ERR_STATE, "st_set_design must precede st_solve_forward_batch");
        CKS(check_source(ms[k], q[k]));
    }
    for (int k = 0; k < count; ++k) {
        cudaSetDevice(ms[k]->device);
        st::launch_rhs(ms[k]->sd, ms[k]->lv[0].g, q[k].kind, q[k].q0, q[k].a, q[k].b, q[k].f, ms[k]->f,
                       ms[k]->stream);
    }
    std::vector<st_status> st(count, ST_OK);
    const st_status r = st::solve_batch(ms.data(), count, false, o, stats, st.data());
    // a failure of the batch itself (argument, CUDA) leaves no state; otherwise per mesh
    const bool hard = !(r == ST_OK || r == ST_ERR_NOT_CONVERGED || r == ST_ERR_NUMERIC);
    for (int k = 0; k < count; ++k) {
        if (hard) st[k] = r;
        ms[k]->have_state = st[k] == ST_OK || st[k] == ST_ERR_NOT_CONVERGED;
        ms[k]->have_adjoint = false;
        if (status) status[k] = st[k];
    }
    return r;
}

st_status st_solve_adjoint_batch(st_mesh* const* m, int count, const st_objective* obj, const st_options* o,
                                 double* phi_out, st_stats* stats, st_status* status) {
    if (!m || !obj || count < 1) return fail(ST_ERR_ARG, "null argument or empty batch");
    std::vector<Mesh*> ms(count);
    for (int k = 0; k < count; ++k) {
        if (!m[k]) return fail(ST_ERR_ARG, "null mesh in the batch");
        ms[k] = M(m[k]);
        CKS(adjoint_rhs(ms[k], &obj[k], phi_out ? &phi_out[k] : nullptr));
    }
    std::vector<st_status> st(count, ST_OK);
    const st_status r = st::solve_batch(ms.data(), count, true, o, stats, st.data());
    const bool hard = !(r == ST_OK || r == ST_ERR_NOT_CONVERGED || r == ST_ERR_NUMERIC);
    for (int k = 0; k < count; ++k) {
        if (hard) st[k] = r;
        ms[k]->have_adjoint = st[k] == ST_OK || st[k] == ST_ERR_NOT_CONVERGED;
        if (status) status[k] = st[k];
    }
    return r;
}

st_status st_sensitivities(st_mesh* m, double* out, size_t count, int mem) {
    if (!m || !out) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    if (!mm->have_adjoint) return fail(ST_ERR_STATE, "st_solve_adjoint must precede st_sensitivities");
    if ((long long)count != mm->design_count) return fail(ST_ERR_ARG, "count must equal the design size");
    cudaSetDevice(mm->device);
    st::launch_sens(mm->sd, mm->op0<double>(), mm->s, mm->lam, mm->gsens, mm->stream);
    cudaError_t e = cudaMemcpyAsync(out, mm->gsens, count * sizeof(double),
                                    mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    mm->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

st_status st_get_state(st_mesh* m, int which, double* out, size_t count, int mem) {
    if (!m || !out) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    if ((long long)count != mm->lv[0].g.nnodes) return fail(ST_ERR_ARG, "count must equal the node count");
    const double* src = which == ST_STATE_T ? mm->s : which == ST_STATE_LAMBDA ? mm->lam
                      : which == ST_STATE_RHS ? mm->f : which == ST_STATE_ADJ_RHS ? mm->adjrhs : nullptr;
    if (!src) return fail(ST_ERR_ARG, "unknown state kind");
    cudaSetDevice(mm->device);
    cudaError_t e = cudaMemcpyAsync(out, src, count * sizeof(double),
                                    mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    mm->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

st_status st_set_state(st_mesh* m, const double* s, size_t count, int mem) {
    if (!m || !s) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    if ((long long)count != mm->lv[0].g.nnodes) return fail(ST_ERR_ARG, "count must equal the node count");
    cudaSetDevice(mm->device);
    cudaError_t e = cudaMemcpyAsync(mm->s, s, count * sizeof(double),
                                    mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    mm->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

// ---- component entry points
static st_status comp_check(Mesh* mm, int level, int precision) {
    if (!mm->have_design) return fail(ST_ERR_STATE, "st_set_design must come first");
    if (level < 0 || level >= (int)mm->lv.size()) return fail(ST_ERR_ARG, "level out of range");
    if (precision != ST_PREC_MIXED && precision != ST_PREC_FP64) return fail(ST_ERR_ARG, "unknown precision");
    cudaSetDevice(mm->device);
    return ST_OK;
}

static st_status finish(Mesh* mm) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(mm->stream);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, cudaGetErrorString(e));
    return ST_OK;
}

st_status st_op_apply(st_mesh* m, int level, int precision, int transpose, const void* x, void* y) {
    if (!m || !x || !y) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, level, precision));
    if (precision == ST_PREC_MIXED) {
        if (level == 0)
            st::launch_apply_l0<float>(mm->sd, mm->op0<float>(), transpose, (const float*)x, (float*)y, mm->stream);
        else
            st::launch_apply_lc<float>(mm->sd, mm->opc<float>(level), transpose, (const float*)x, (float*)y, mm->stream);
    } else {
        if (level == 0)
            st::launch_apply_l0<double>(mm->sd, mm->op0<double>(), transpose, (const double*)x, (double*)y, mm->stream);
        else
            st::launch_apply_lc<double>(mm->sd, mm->opc<double>(level), transpose, (const double*)x, (double*)y,
                                        mm->stream);
    }
    return finish(mm);
}

st_status st_op_diag(st_mesh* m, int level, int precision, void* d) {
    if (!m || !d) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, level, precision));
    if (precision == ST_PREC_MIXED) {
        if (level == 0)
            st::launch_diag_l0<float>(mm->sd, mm->op0<float>(), (float*)d, false, mm->stream);
        else
            st::launch_diag_lc<float>(mm->sd, mm->opc<float>(level), (float*)d, false, mm->stream);
    } else {
        if (level == 0)
            st::launch_diag_l0<double>(mm->sd, mm->op0<double>(), (double*)d, false, mm->stream);
        else
            st::launch_diag_lc<double>(mm->sd, mm->opc<double>(level), (double*)d, false, mm->stream);
    }
    return finish(mm);
}

st_status st_restrict(st_mesh* m, int level, int precision, const void* rf, void* rc) {
    if (!m || !rf || !rc) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, level, precision));
    if (level + 1 >= (int)mm->lv.size()) return fail(ST_ERR_ARG, "no coarser level");
    const st::LevelH& F = mm->lv[level];
    const st::LevelH& C = mm->lv[level + 1];
    if (precision == ST_PREC_MIXED)
        st::launch_restrict<float>(F.g, C.g, F.to_next, mm->sd, (const float*)rf, (float*)rc, mm->stream);
    else
        st::launch_restrict<double>(F.g, C.g, F.to_next, mm->sd, (const double*)rf, (double*)rc, mm->stream);
    return finish(mm);
}

st_status st_prolong(st_mesh* m, int level, int precision, const void* xc, void* xf) {
    if (!m || !xc || !xf) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, level, precision));
    if (level + 1 >= (int)mm->lv.size()) return fail(ST_ERR_ARG, "no coarser level");
    const st::LevelH& F = mm->lv[level];
    const st::LevelH& C = mm->lv[level + 1];
    if (precision == ST_PREC_MIXED)
        st::launch_prolong<float>(F.g, C.g, F.to_next, mm->sd, (const float*)xc, (float*)xf, mm->stream);
    else
        st::launch_prolong<double>(F.g, C.g, F.to_next, mm->sd, (const double*)xc, (double*)xf, mm->stream);
    return finish(mm);
}

st_status st_smooth(st_mesh* m, int level, int precision, int transpose, const void* b, void* x, int steps,
                    int zero_init) {
    if (!m || !b || !x) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, level, precision));
    if (steps < 1 || steps > st::kMaxSmooth) return fail(ST_ERR_ARG, "steps must be in [1, 16]");
    if (precision == ST_PREC_MIXED) return smooth_entry<float>(mm, level, transpose, b, x, steps, zero_init);
    return smooth_entry<double>(mm, level, transpose, b, x, steps, zero_init);
}

st_status st_vcycle(st_mesh* m, int precision, int transpose, const void* b, void* x) {
    if (!m || !b || !x) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, 0, precision));
    if (precision == ST_PREC_MIXED) return vcycle_entry<float>(mm, transpose, b, x);
    return vcycle_entry<double>(mm, transpose, b, x);
}

st_status st_level_elements(st_mesh* m, int level, double* out, size_t count) {
    if (!m || !out) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, level, ST_PREC_FP64));
    if (level < 1) return fail(ST_ERR_ARG, "level 0 is matrix free");
    const long long want = mm->lv[level].nstore * st::nvals(mm->sd);
    if ((long long)count != want) return fail(ST_ERR_ARG, "count must be " + std::to_string(want));
    CK(cudaMemcpyAsync(out, mm->lv[level].e64, want * sizeof(double), cudaMemcpyDeviceToHost, mm->stream));
    return finish(mm);
}

st_status st_apply_timer(st_mesh* m, int enable) {
    if (!m) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    if (mm->device >= 0) cudaSetDevice(mm->device);
    CK(cudaStreamSynchronize(mm->stream));
    if (enable) {
        for (cudaEvent_t& e : mm->at_ev)
            if (!e) CK(cudaEventCreate(&e));
        mm->at_ms = 0.0;
        mm->at_launches = 0;
    }
    mm->at_pending = false;
    if ((enable != 0) != mm->at_on) mm->drop_graphs();  // recapture with or without the event nodes
    mm->at_on = enable != 0;
    return ST_OK;
}

st_status st_apply_timer_read(st_mesh* m, double* total_ms, long long* launches) {
    if (!m || !total_ms || !launches) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    *total_ms = mm->at_ms;
    *launches = mm->at_launches;
    return ST_OK;
}

st_status st_coarse_inverse(st_mesh* m, double* out, size_t count) {
    if (!m || !out) return fail(ST_ERR_ARG, "null argument");
    Mesh* mm = M(m);
    CKS(comp_check(mm, 0, ST_PREC_FP64));
    if (mm->coarse_iter) return fail(ST_ERR_STATE, "the coarsest level is solved iteratively (no dense inverse)");
    const long long n = mm->lv.back().g.nnodes;
    if ((long long)count != n * n) return fail(ST_ERR_ARG, "count must be n*n of the coarsest level");
    CK(cudaMemcpyAsync(out, mm->Ainv, n * n * sizeof(double), cudaMemcpyDeviceToHost, mm->stream));
    return finish(mm);
}

}  // extern "C"
