// Internal declarations shared by the CUDA translation units of the space-time solver.
//
// Geometry, operator descriptors and launch wrappers.  Device code lives in
// k_ops.cu (operator applies, transfers, smoother, Krylov kernels) and
// k_setup.cu (design cast, Galerkin coarse operators, coarsest inverse,
// source, objective, sensitivities); host orchestration in solver.cu.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/st.h"

namespace st {

// Programmatic dependent launch.  Every kernel of the library starts with pdl_enter(): it
// waits until the previous kernel in the stream has completed and its memory is visible, then
// lets the next kernel be scheduled.  Launched through launch_pdl, the next kernel's launch and
// block set-up overlap the tail of the current one (also inside captured graphs); launched
// without the attribute, both instructions return at once.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
#endif

extern bool g_pdl;  // environment ST_PDL=0 turns the launch attribute off
// Set by the calling thread while it captures the bodies of conditional graph nodes: launches
// then carry no programmatic-serialization attribute (plain stream order inside the bodies).
extern thread_local bool g_no_pdl;

template <typename... KP, typename... A>
inline void launch_pdl(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (g_pdl && !g_no_pdl) ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

constexpr int kMaxLevels = 40;
constexpr int kMaxSmooth = 16;     // Jacobi-GMRES steps per smoothing call
constexpr int kMaxRestart = 32;    // FGMRES restart length
constexpr int kMaxBlocks = 4096;   // blocks of a reducing kernel (partial-sum buffer size)
constexpr int kMaxCoarse = 4096;   // largest coarsest level (dense inverse)
constexpr int kRedQ = 32;          // partial sums per block (>= kMaxRestart, kMaxSmooth)

// Node/element geometry of one level.  Spatial axes are x, y, z (z unused in 2D);
// nodes are ordered ((n * nz1 + k) * ny1 + j) * nx1 + i.
struct Geom {
    int nx1, ny1, nz1, nt1;        // node counts per axis (nz1 = 1 in 2D)
    int nex, ney, nez, net;        // element counts (nez = 1 in 2D)
    long long plane;               // nodes per time plane
    long long nnodes;
    long long sp_elems;            // spatial elements per time slab
    double h[3];                   // spatial element sizes
    double dt;
    int bc;                        // ST_BC_*
    int face;                      // patch face axis (0: x = 0, 1: y = 0)
    int plo[3], phi[3];            // patch node range per spatial axis (inclusive)
    int march_blocks;              // thread-block budget of the time-marching kernels (<= 0: the default, 912)
};

// Modified SIMP parameters (C = C_ins + dC g^p_c, k = k_ins + dk g^p_k).
struct Simp {
    double C_ins, dC, k_ins, dk;
    int p_c, p_k;
};

// Level-0 (fine) operator: matrix free from the design.  Element matrix
// J_e = C_e (D_t (x) M_x) + k_e (M_t (x) K_x); M_x and K_x entries depend only on
// which local bits differ, so they are tabulated by (a ^ b).
template <typename T>
struct OpL0 {
    Geom g;
    const double* g64;             // FP64 design (used when T = double)
    const __nv_bfloat16* g16;      // BF16 design (used when T = float)
    int tc;                        // 1: extruded design (per spatial element)
    Simp simp;
    T mxd[8], kxd[8];              // M_x, K_x by (a ^ b) over spatial bits
    T dt6;                         // dt / 6 (time mass scale)
    const T* st_coef[2];           // 27-point stencils [class][27][P] (forward, transposed), or null
    const unsigned char* st_dir;   // spatial prescribed flags when stencils are present
};

// Coarse operator (levels >= 1): element matrices in block form, 4 symmetric
// spatial blocks (a_t, b_t) packed as upper triangles; extruded designs keep two
// versions per spatial element (first slab, other slabs).
template <typename T>
struct OpLc {
    Geom g;
    const T* elem;
    int tc;
    const T* st_coef[2];           // as in OpL0
    const unsigned char* st_dir;
    const float* x3st;             // extruded 3-D designs, FP32 path: stencils MC, KD [54][P], or null
    float x3tw[8];                 // the level's time matrices D_t, M_t ([a_t][b_t]) for x3st
    const float* x2blk;            // space-time 2-D designs, space-coarsened levels: M, K rows [slab][elem][32]
};

// Per-call smoother state (device), in the arithmetic type T of its multigrid (float for
// the mixed V-cycle: FP64 arithmetic is a slow path on this GPU).  SmState is the opaque
// storage (large enough for either type); kernels view it as SmStateT<T>.
template <typename T>
struct SmStateT {
    T H[(kMaxSmooth + 1) * kMaxSmooth];   // Hessenberg matrix, row-major
    T R[(kMaxSmooth + 1) * kMaxSmooth];   // after Givens rotations
    T s[kMaxSmooth + 1];                  // basis scales 1 / ||u_j||
    T cs[kMaxSmooth], sn[kMaxSmooth], g[kMaxSmooth + 1];
    T coef[kMaxSmooth];                   // y_j s_j of the final update
    T beta;
    int kdim;
    int stop;
    // Restarted use as a solver (the coarsest-level Jacobi-GMRES): rtol_rel > 0 stops the
    // Arnoldi process once the residual estimate reaches atol = rtol_rel ||b|| (atol < 0:
    // taken from the next start) and skips every later restart cycle.  0 for the smoother.
    T rtol_rel;
    T atol;
};

struct alignas(16) SmState {
    unsigned char bytes[sizeof(SmStateT<double>)];
};

template <typename T>
__host__ __device__ inline SmStateT<T>* smt(SmState* s) {
    return reinterpret_cast<SmStateT<T>*>(s);
}
template <typename T>
__host__ __device__ inline const SmStateT<T>* smt(const SmState* s) {
    return reinterpret_cast<const SmStateT<T>*>(s);
}

// FGMRES state (device).
struct FgState {
    double H[(kMaxRestart + 1) * kMaxRestart];
    double h1[kMaxRestart + 1];
    double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1];
    double beta;
    double res_est;
    double nrm;                    // scratch scalar result
    int breakdown;
    int bad;                       // NaN/Inf seen
    // graph-resident restart cycles (no host synchronisation per iteration)
    int its;                       // outer iterations of the solve so far
    int kdone;                     // iterations completed in the current restart cycle
    int cont;                      // 1: the cycle takes another iteration
};

struct RedBuf {
    double* part;                  // [kMaxBlocks][kRedQ]
    unsigned* counter;
};

template <typename T>
struct Basis {
    T* u[kMaxSmooth + 1];
};

// Basis pointers passed by value to the streaming kernels (smoother or FGMRES basis).
template <typename T>
struct Ptrs {
    T* p[kMaxRestart + 1];
};

struct LaunchCfg {
    dim3 grid, block;
};

LaunchCfg node_cfg(const Geom& g);

// Kernel-launch accounting (st_kernel_launches): n launches queued on s; launches
// recorded into a graph under capture are counted when the graph is replayed.
void note_launch(cudaStream_t s, long long n = 1);
void note_graph_launch(long long kernels);

// ---------------------------------------------------------------- launch wrappers
// All take the spatial dimension sd (2|3) and dispatch to templates.
// Operator applies: y = A x (transpose: A^T x).
template <typename T>
void launch_apply_l0(int sd, const OpL0<T>& op, bool tr, const T* x, T* y, cudaStream_t s);
template <typename T>
void launch_apply_lc(int sd, const OpLc<T>& op, bool tr, const T* x, T* y, cudaStream_t s);
template <typename T>
void launch_diag_l0(int sd, const OpL0<T>& op, T* dinv, bool invert, cudaStream_t s);
template <typename T>
void launch_diag_lc(int sd, const OpLc<T>& op, T* dinv, bool invert, cudaStream_t s);
// r = b - A x
template <typename T>
void launch_residual(int sd, int lvl, const OpL0<T>& o0, const OpLc<T>& oc, bool tr, const T* b,
                     const T* x, T* r, cudaStream_t s);
// transfers between level (fine geometry gf) and level+1 (gc); kind 0 space, 1 time, 2 full
template <typename T>
void launch_restrict(const Geom& gf, const Geom& gc, int kind, int sd, const T* rf, T* rc, cudaStream_t s);
template <typename T>
void launch_prolong(const Geom& gf, const Geom& gc, int kind, int sd, const T* xc, T* xf, cudaStream_t s);

// Jacobi-GMRES smoother on one level (w2: second scratch vector for the fused FP32 steps).
// `sweeps` damped Jacobi sweeps x += omega D^-1 (b - A x) (A^T if tr) on level lvl, the first
// one from x = 0 when zero_init (then x = omega D^-1 b); r is scratch for the residual.
template <typename T>
void launch_jacobi_smooth(int sd, int lvl, const OpL0<T>& o0, const OpLc<T>& oc, bool tr, const T* b, T* x,
                          const T* dinv, T* r, int sweeps, bool zero_init, T omega, cudaStream_t s);
template <typename T>
void launch_smooth(int sd, int lvl, const OpL0<T>& o0, const OpLc<T>& oc, bool tr, const T* b, T* x,
                   const T* dinv, Basis<T> U, T* w, T* w2, int steps, bool zero_init, SmState* st, RedBuf rb,
                   cudaStream_t s, cudaEvent_t* apply_ev = nullptr, const T* scaled_stencil = nullptr);
// Interior-class stencils of a stencil level with the Jacobi scaling of the neighbour folded
// in: sc[o][k][p] = st[o][1][k][p] dinv(n_ref, q_k(p)), identity rows d(p) at prescribed
// spatial nodes (k_march.cu).
template <typename T>
void launch_stencil_scale(const Geom& g, const T* st, const T* dinv, const unsigned char* dir, T* sc,
                          cudaStream_t s);
// Jacobi diagonal (or its inverse) of a stencil level from the stencil's centre coefficients
// (k_march.cu); coef is the forward-orientation class stencil set [class][27][P].
template <typename T>
void launch_stencil_diag(const Geom& g, const T* coef, const unsigned char* dir, T* d, bool invert, cudaStream_t s);
// One Arnoldi step j of the smoother on a stencil level as one kernel (k_smstep.cuh): the
// update u_j = s_{j-1} w_{j-1} - sum H[q][j-1] s_q u_q (j >= 1), w_j = A D^-1 u_j with the
// scaled interior stencil sc, and the dots (w_j, u_q), q <= j, with ||u_j||^2.  Instantiated for
// float (the mixed V-cycle); the FP64 V-cycle uses the separate kernels.
template <typename T>
void launch_sm_step(const Geom& g, const T* sc, const T* coef, const unsigned char* dir, const T* dinv,
                    const Ptrs<T>& U, const T* wprev, T* wout, int j, int steps, SmState* st, RedBuf rb,
                    cudaStream_t s);
// Whether the step kernel can run the sweep: 16-byte aligned vectors, fewer than 2^31 nodes, at
// least 64 per plane, and every step's ring within one block's shared memory.
template <typename T>
bool sm_step_aligned(const Ptrs<T>& U, int steps, const T* w, const T* w2, long long nnodes, long long plane);
extern bool g_smstep;  // environment ST_SMSTEP=0: separate apply, dot and update kernels instead
extern bool g_l0st;   // environment ST_L0ST=0: level-0 space-time rows by the node-parallel kernels instead
// Level-0 rows of a space-time 2-D design in FP32 as time-marching kernels (k_l0st.cu): mode 0
// w = A D^-1 u (smoother apply), 1 r = b - A x, 2 u_0 = b - A x with ||u_0||^2 (smoother
// start), 3 y = A x.  Usable when the design is per space-time element, the level has fewer than 2^31
// nodes and elements and at least 64 nodes per plane, and every vector (null entries skipped)
// starts on a 16-byte boundary.
bool l0st_usable(const OpL0<float>& op, const void* const* vecs, int nvec);
void launch_l0st(int mode, bool tr, const OpL0<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s);
// The same rows for extruded 3-D designs (k_l0x3.cu), usable for those designs with at least 64
// nodes per plane, fewer than 2^31 nodes and 16-byte aligned vectors.
bool l0x3_usable(const OpL0<float>& op, const void* const* vecs, int nvec);
void launch_l0x3(int mode, bool tr, const OpL0<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s);
// Coarse levels of extruded 3-D designs (k_l0x3.cu): the same marching rows from each node's
// two extracted stencils (op.x3st) and the level's time matrices; k_x3_stencil extracts them
// from the FP64 element blocks once per design.
bool lcx3_usable(const OpLc<float>& op, const void* const* vecs, int nvec);
void launch_lcx3(int mode, bool tr, const OpLc<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s);
void launch_x3_stencil(const OpLc<double>& op, const double Dt[4], const double Mt[4], float* out, cudaStream_t s);
// Space-coarsened levels of space-time 2-D designs (k_lcst.cu): marching rows from each
// (slab, element)'s M and K rows (op.x2blk), extracted once per design by k_x2_blocks.
bool lcst_usable(const OpLc<float>& op, const void* const* vecs, int nvec);
void launch_lcst(int mode, bool tr, const OpLc<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s);
void launch_x2_blocks(const OpLc<double>& op, float* out, cudaStream_t s);
// FP64 level-0 rows of the outer FGMRES for space-time 2-D and extruded 3-D designs as marching
// kernels (k_fg_march.cu): mode 0 w = J z (z copied into zstore when given), mode 1
// r = f - J x with ||r||^2 into the FGMRES state.  Usable for those designs with at least 64
// nodes per plane, fewer than 2^31 nodes and 16-byte aligned vectors.
bool fg_march_usable(int sd, const OpL0<double>& op, const void* const* vecs, int nvec);
template <typename TZ>
void launch_fg_march(int sd, int mode, bool tr, const OpL0<double>& op, const TZ* z, TZ* zstore, const double* f,
                     double* out, FgState* fs, RedBuf rb, cudaStream_t s);
// Fused FP32 Arnoldi step j -> j+1 on a stencil level (k_arnoldi.cu).
void launch_arnoldi(const Geom& g, const float* coef, const unsigned char* dir, const float* dinv,
                    const Ptrs<float>& U, const float* w_in, float* w_out, int j, SmState* st, RedBuf rb,
                    cudaStream_t s);

// Coarsest solve x = Ainv b (or Ainv^T b).
template <typename T>
void launch_coarse_solve(const double* Ainv, int n, bool tr, const T* b, T* x, cudaStream_t s);

// ---- FGMRES (FP64 outer) kernels; TZ is the multigrid vector type
template <typename TZ>
void launch_fg_apply_dots(int sd, const OpL0<double>& op, bool tr, const TZ* z, TZ* zstore,
                          double* w, double* const* V, int j, FgState* fs, RedBuf rb, cudaStream_t s);
void launch_fg_update_dots(const Geom& g, double* w, double* const* V, int j, int pass, FgState* fs,
                           RedBuf rb, cudaStream_t s);
template <typename TZ>
void launch_fg_normalize(const Geom& g, const double* w, double* vnext, TZ* bmg, int j, FgState* fs,
                         cudaStream_t s);
template <typename TZ>
void launch_fg_update_x(const Geom& g, double* x, TZ* const* Z, int k, FgState* fs, cudaStream_t s);
// The same with k read on the device (fs->kdone), for graph-resident restart cycles.
template <typename TZ>
void launch_fg_update_x_dev(const Geom& g, double* x, TZ* const* Z, int m, FgState* fs, cudaStream_t s);
// Graph-resident FGMRES cycle control (conditional graph nodes, Sec. 3.2 outer solve):
// begin: iterate iff beta > tol, finite, its < max_it (sets the WHILE condition hw, kdone = 0);
// setj: SWITCH index hs = kdone (the iteration about to run); check (after iteration j's
// Givens rotation): its += 1, kdone = j + 1, cont = not (NaN, res_est <= tol, breakdown,
// its >= max_it, j + 1 == m); loop: hw = cont.
void launch_fg_begin(FgState* fs, double tol, int max_it, cudaGraphConditionalHandle hw, cudaStream_t s);
void launch_fg_setj(const FgState* fs, cudaGraphConditionalHandle hs, cudaStream_t s);
void launch_fg_check(FgState* fs, int j, double tol, int max_it, int m, cudaStream_t s);
void launch_fg_loop(const FgState* fs, cudaGraphConditionalHandle hw, cudaStream_t s);
void launch_fg_residual(int sd, const OpL0<double>& op, bool tr, const double* f, const double* x,
                        double* r, FgState* fs, RedBuf rb, cudaStream_t s);
template <typename TZ>
void launch_fg_start(const Geom& g, double* v0, TZ* bmg, FgState* fs, cudaStream_t s);
void launch_dot64(const Geom& g, const double* a, const double* b, double* out, RedBuf rb, cudaStream_t s);
void launch_mask_copy(int sd, const Geom& g, const double* src, double* dst, cudaStream_t s);

// ---- streaming Krylov kernels (k_stream.cu)
// dots (w, U_q) for q < nq -> smoother column j (fin 0) or FGMRES first projection (fin 1)
template <typename T>
void launch_dots(long long n, const T* w, const Ptrs<T>& U, int nq, int j, int fin, void* state, RedBuf rb,
                 cudaStream_t s);
// y = a w - sum_{q<=j} c_q U_q; mode 0 smoother step, 1 / 2 FGMRES CGS2 passes (y = w)
template <typename T>
void launch_update(long long n, T* w, T* y, const Ptrs<T>& U, int j, int steps, int mode, void* state, RedBuf rb,
                   cudaStream_t s);
template <typename T>
void launch_sm_combine(long long n, T* x, const T* dinv, const Ptrs<T>& U, int steps, bool zero_init,
                       const SmState* st, cudaStream_t s);
template <typename T>
void launch_sm_norm(long long n, const T* b, int steps, SmState* st, RedBuf rb, cudaStream_t s);
template <typename TZ>
void launch_fg_combine(long long n, double* x, const Ptrs<TZ>& Z, int k, const FgState* fs, cudaStream_t s);

// ---- setup kernels
void launch_design_cast(const double* in, double* g64, __nv_bfloat16* g16, long long n, int* bad, cudaStream_t s);
void launch_build_from_l0(int sd, const OpL0<double>& f0, const Geom& gc, int kind, int tc, double* elem_c,
                          cudaStream_t s);
void launch_build_from_lc(int sd, const OpLc<double>& fc, const Geom& gc, int kind, double* elem_c,
                          cudaStream_t s);
void launch_to_float(const double* in, float* out, long long n, cudaStream_t s);
// Coarsest-level Jacobi-GMRES (k_stream.cu): set the relative tolerance of the solver state,
// and convert the level vectors between the V-cycle precision and FP64.
template <typename T>
void launch_cg_begin(SmState* st, double rtol, cudaStream_t s);
template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, long long n, cudaStream_t s);
void launch_dense_assemble(int sd, int lvl, const OpL0<double>& o0, const OpLc<double>& oc, double* A,
                           cudaStream_t s);
// Gauss-Jordan inverse of the dense n x n matrix A (result in A, B scratch); *err = 1 on a zero
// pivot.  One cooperative kernel eliminating 8 (or 4) pivots per step with two bounded grid
// barriers per step (PR: 8 n doubles of scratch, bar: barrier counter, *tmo = 1 if a barrier wait gave
// up), else one launch per pivot.
void launch_gauss_jordan(double* A, double* B, double* pinv, double* PR, int n, int* err, unsigned* bar, int* tmo,
                         cudaStream_t s);
void launch_rhs(int sd, const Geom& g, int kind, double q0, double a, double b, double f, double* out,
                cudaStream_t s);
void launch_pnorm(int sd, const Geom& g, const double* s, int P, double* rhs, double* phi, RedBuf rb,
                  double* scratch, cudaStream_t st);
void launch_sens(int sd, const OpL0<double>& op, const double* s, const double* lam, double* out,
                 cudaStream_t st);
// 27-point stencils of a time-constant 2-D level (from level 0 or from stored element blocks)
void launch_stencil_build(int lvl, const OpL0<double>& o0, const OpLc<double>& oc, double* st64, float* st32,
                          unsigned char* dir, cudaStream_t s);

// ---- PDE filter and projection (k_filter.cu, Sec. 3.3.2)
// y = (M_f + K_f) x with the class table tab (3^(SD+1) classes x 3^(SD+1) offsets), or dinv = the
// inverse diagonal when dinv is given; rhs: (T gamma) = scale * sum of the adjacent elements'
// values; mean: element means of a nodal field; CG vector updates (z and p of cg_zp may be the
// same vector); projection H and H'.
void launch_filter_apply(int sd, const Geom& g, const double* tab, const double* x, double* y, double* dinv,
                         cudaStream_t s);
void launch_filter_rhs(int sd, const Geom& g, const double* gam, double scale, double* out, cudaStream_t s);
void launch_filter_mean(int sd, const Geom& g, const double* psi, double* out, cudaStream_t s);
void launch_cg_xr(long long n, double a, const double* p, const double* q, double* x, double* r, cudaStream_t s);
void launch_cg_zp(long long n, double b, const double* dinv, const double* r, double* z, double* p, cudaStream_t s);
void launch_cg_p(long long n, double b, const double* z, double* p, cudaStream_t s);
void launch_heaviside(long long n, const double* in, double* out, double* dout, double beta, double eta,
                      cudaStream_t s);

// element storage sizes
inline int nsp(int sd) { return 1 << sd; }
inline int nsym(int sd) { return nsp(sd) * (nsp(sd) + 1) / 2; }
inline int nvals(int sd) { return 4 * nsym(sd); }

}  // namespace st

#define ST_CUDA_LAUNCH_CHECK() \
    do {                       \
    } while (0)
