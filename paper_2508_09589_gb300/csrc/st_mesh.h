// Mesh object behind the st_mesh handle: hierarchy, design, device buffers and the
// per-precision multigrid workspaces.
#pragma once

#include <vector>

#include "st_internal.h"
#include "st_vtail.h"

namespace st {

st_status fail(st_status code, const std::string& msg);
long long kernel_launches();
extern thread_local std::string g_last_error;

struct LevelH {
    Geom g;
    int to_next = -1;          // 0 space, 1 time, 2 both, -1 coarsest
    long long nstore = 0;      // stored element matrices (levels >= 1)
    double* e64 = nullptr;     // FP64 element blocks
    float* e32 = nullptr;      // FP32 copy for the mixed V-cycle
    double* st64 = nullptr;    // 27-point stencils [orientation][class][27][P] (extruded, 2-D)
    float* st32 = nullptr;
    unsigned char* sdir = nullptr;
    float* x3st = nullptr;     // extruded 3-D designs, levels >= 1 with n_t >= 2: stencils MC, KD [54][P]
    float x3tw[8] = {};        // and the level's time matrices D_t, M_t ([a_t][b_t])
    float* x2blk = nullptr;    // space-time 2-D designs, levels reached by space coarsening only: M, K rows
};

template <typename T>
struct MGWork {
    VTail<T>* d_vt = nullptr;      // persistent coarse-tail descriptor (device)
    long long vt_version = -1;
    int steps_uploaded = -1;
    bool ready = false;
    int nbasis = 0;
    long long dinv_version = -1;
    std::vector<T*> b, x, r, w, w2, dinv;
    std::vector<T*> sc;            // stencil levels: interior stencils with the Jacobi scaling folded in
    std::vector<Basis<T>> U;
};

struct Mesh {
    st_mesh_desc desc{};
    int sd = 2;
    int device = -1;
    cudaStream_t stream = nullptr;
    cudaStream_t own = nullptr;
    bool own_stream = false;
    std::vector<LevelH> lv;

    // design
    int layout = ST_DESIGN_EXTRUDED;
    int storage_tc = -1;
    long long design_count = 0;
    long long design_version = 0;
    double* gin = nullptr;
    double* g64 = nullptr;
    __nv_bfloat16* g16 = nullptr;
    double* gsens = nullptr;
    bool have_design = false, have_state = false, have_adjoint = false;

    // coarsest level: dense inverse, or the iterative Jacobi-GMRES solve (coarse_iter) with
    // its FP64 vectors, restart length cg_m and cycle count
    bool coarse_iter = false;
    int cg_m = 16;
    int cg_cycles = 0;
    double* cg_b = nullptr;
    double* cg_x = nullptr;
    double* cg_dinv = nullptr;
    double* cg_w = nullptr;
    double* cg_w2 = nullptr;
    Basis<double> cg_U{};
    SmState* d_smc = nullptr;
    long long cg_dinv_version = -1;
    template <typename T>
    void coarse_gmres(bool tr);
    double* Ainv = nullptr;
    double* Awork = nullptr;
    double* gjpr = nullptr;        // scratch of the blocked inverse (8 rows of the coarsest size)
    double* pinv = nullptr;
    int* d_err = nullptr;

    // FP64 vectors
    double* f = nullptr;
    double* s = nullptr;
    double* lam = nullptr;
    double* adjrhs = nullptr;
    double* fg_w = nullptr;
    std::vector<double*> V;
    std::vector<float*> Z32;
    std::vector<double*> Z64;

    MGWork<float> w32;
    MGWork<double> w64;

    int vt_first = -1;             // first level of the persistent coarse tail (-1: none)
    bool vt_failed = false;        // its cooperative launch was refused: one launch per phase instead
    unsigned vt_spin_limit = 1u << 24;  // grid-barrier polls before a wait gives up (ST_VTAIL_SPIN_LIMIT)
    long long vt_max_nodes = 0;    // persistent coarse tail off by default (ST_VTAIL_NODES enables it)
    long long ws_version = 0;      // bumped when multigrid buffers move
    unsigned* d_bar = nullptr;
    unsigned long long* vt_trace = nullptr;
    double* vt_part = nullptr;
    SmState* d_sm = nullptr;
    FgState* d_fg = nullptr;
    FgState* h_fg = nullptr;
    RedBuf rb{};
    double* d_scalar = nullptr;

    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
    int gsteps[4] = {0, 0, 0, 0};
    long long gversion[4] = {-1, -1, -1, -1};
    long long gkernels[4] = {0, 0, 0, 0};

    // opt-in per-level timing of eager V-cycles (environment ST_LEVEL_TIMING=1), printed at exit
    bool level_timing = false;
    std::vector<cudaEvent_t> tev;
    std::vector<double> tacc;      // [level][phase]: pre-smooth, down-transfer, post-smooth+prolong
    int tcycles = 0;
    bool capturing = false;

    // opt-in CUDA-event timing of every level-0 smoother operator apply (st_apply_timer):
    // event pairs [sweep][step] recorded around the launches (event nodes inside captured
    // V-cycles) and read after the host synchronisation that follows each V-cycle
    bool at_on = false;
    bool at_pending = false;
    int at_steps = 0;
    cudaEvent_t at_ev[4 * kMaxSmooth] = {};
    double at_ms = 0.0;
    long long at_launches = 0;
    void timer_collect();

    // PDE filter scratch: 7 nodal vectors (rhs, x, r, z, p, q, D^-1), 2 element fields, the
    // class table and 4 scalars
    double* fbuf = nullptr;
    long long fbuf_len = 0;

    std::vector<void*> allocs;
    std::vector<size_t> alloc_sizes;
    long long bytes_held = 0;

    ~Mesh();
    st_status alloc(void** p, size_t bytes);
    void release(void* p);
    void drop_graphs();
    st_status ensure_level_storage();

    template <typename T>
    OpL0<T> op0() const;
    template <typename T>
    OpLc<T> opc(int l) const;
    template <typename T>
    MGWork<T>& work();
    template <typename T>
    st_status ensure_mg(int steps);
    template <typename T>
    st_status upload_vtail(int steps);
    template <typename T>
    void smooth(int l, bool tr, bool zero_init, int steps);
    template <typename T>
    void vcycle_rec(int l, bool tr, int steps);
    template <typename T>
    st_status vcycle(bool tr, int steps, bool graphs);
    template <typename T>
    st_status fgmres(bool tr, const double* rhs, double* x, const st_options& o, st_stats* stats);
    // FGMRES storage (V: m + 1 FP64 vectors, Z: m vectors of the preconditioner's precision)
    template <typename T>
    st_status ensure_krylov(int m, int steps);
    // Graph-resident restart cycle: captures into graph G (a branch with no dependencies) the
    // residual, the cycle start, a WHILE node whose body holds the V-cycle and a SWITCH over the
    // iteration index with the Arnoldi kernels of each iteration, the solution update and the
    // final residual.  cs: three capture streams.  *per_iter and *fixed count its kernels.
    template <typename T>
    st_status capture_cycle(cudaGraph_t G, cudaStream_t* cs, bool tr, const st_options& o, double tol,
                            const double* rhs, double* x, long long* per_iter, long long* fixed);
};

// Forward (adjoint = false) or adjoint solves of several meshes of one device whose right-hand
// sides are assembled, as graph-resident FGMRES restart cycles: one graph holds every mesh's
// cycle as an independent branch and one launch advances all of them by a whole restart cycle
// (iterations, convergence tests and the stop decision on the device); the host synchronises
// once per cycle.  The graph runs on the first mesh's stream.
st_status solve_batch(Mesh* const* ms, int n, bool adjoint, const st_options* op, st_stats* stats,
                      st_status* status);

// PDE filter of an element field (Sec. 3.3.2) on the mesh's geometry (one slab for an extruded
// field), by Jacobi-preconditioned CG; *iters receives the iterations.
st_status filter(Mesh* m, const double* in, double* out, size_t count, int mem, double rx, double rt, double rtol,
                 int max_it, int* iters);

// the Mesh behind a C-ABI handle
Mesh* mesh_of(st_mesh* m);

// the bodies of st_create_mesh, st_set_design and the forward (adjoint = false) or adjoint solve
// of the right-hand side already in m->f (m->adjrhs), from the state in m->s (m->lam) when
// o->warm_start is set
st_status create_mesh(const st_mesh_desc* d, Mesh** out);
st_status set_design(Mesh* m, const double* gamma, int layout, size_t count, int mem);
st_status solve(Mesh* m, bool adjoint, const st_options* op, st_stats* stats);

}  // namespace st
