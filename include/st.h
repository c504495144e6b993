/*
 * st.h -- C ABI of the GB300 space-time heat-conduction solver.
 *
 * The library solves the all-at-once system J s = f of the stabilised
 * continuous-Galerkin space-time finite-element discretisation of transient
 * heat conduction (arXiv 2508.09589, Sec. 3.1: weak form with time artificial
 * diffusion k_ad = C dt / 2, trilinear elements on a regular space-time mesh,
 * all nodal temperatures in one vector), with capacity C and conductivity k
 * interpolated from a density design by modified SIMP (Sec. 2.2).  The solver
 * is flexible GMRES (FP64) preconditioned by a space-time multigrid V-cycle
 * with semi-coarsening by Algorithm 1, Galerkin coarse operators, trilinear
 * transfers and Jacobi-GMRES smoothing (Sec. 3.2), run in FP32 ("mixed") or
 * FP64.  The adjoint system J^T Lambda = (d phi/d s)^T and the per-element
 * sensitivities of Sec. 3.3.3 use the same hierarchy.
 *
 * Conventions
 *  - Every call returns st_status; 0 is success, negative values are errors.
 *    No call aborts the process.  st_last_error() returns a message for the
 *    last failure on the calling thread.
 *  - Node arrays are ordered with x fastest and time slowest:
 *    index = ((n * (nz+1) + k) * (ny+1) + j) * (nx+1) + i  (nz = 0 in 2D).
 *  - Element arrays use the same order over element indices; an extruded
 *    (time-constant) design holds only the spatial elements.
 *  - Pointer arguments tagged with a `mem` argument are host pointers when
 *    mem == ST_MEM_HOST and device pointers (on the mesh's device) when
 *    mem == ST_MEM_DEVICE.  The caller always owns these buffers; the library
 *    copies inputs and writes outputs, and never keeps the pointer.
 *  - All device memory used by a mesh is owned by the mesh and released by
 *    st_destroy_mesh.  Work is queued on the mesh's stream (st_set_stream);
 *    calls that return host results synchronise that stream.
 *  - A mesh must be used from one thread at a time.
 */
#ifndef ST_H
#define ST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int st_status;
#define ST_OK 0
#define ST_ERR_ARG (-1)            /* invalid argument (size, kind, null pointer) */
#define ST_ERR_OOM (-2)            /* device allocation failed */
#define ST_ERR_NOT_CONVERGED (-3)  /* rtol not reached within max_it; best iterate kept */
#define ST_ERR_NUMERIC (-4)        /* NaN/Inf or a zero pivot was detected */
#define ST_ERR_TIMEOUT (-5)        /* a bounded wait gave up */
#define ST_ERR_CUDA (-6)           /* a CUDA runtime call failed */
#define ST_ERR_BUSY (-7)           /* request refused by admission control */
#define ST_ERR_STATE (-8)          /* call out of order (e.g. solve before set_design) */
#define ST_ERR_NOT_FOUND (-9)      /* unknown ticket */
#define ST_ERR_CANCELLED (-10)     /* the request was cancelled before it was admitted */

enum { ST_BC_PATCH_LEFT = 0, ST_BC_PATCH_BOTTOM = 1, ST_BC_ALL_WALLS = 2, ST_BC_NONE = 3 };
enum { ST_DESIGN_EXTRUDED = 0, ST_DESIGN_SPACETIME = 1 };
enum { ST_MEM_HOST = 0, ST_MEM_DEVICE = 1 };
enum { ST_PREC_MIXED = 0, ST_PREC_FP64 = 1 };
enum { ST_SRC_UNIFORM = 0, ST_SRC_SIN_T = 1, ST_SRC_GAUSSIAN = 2 };
enum { ST_OBJ_COMPLIANCE = 0, ST_OBJ_PNORM = 1 };
enum { ST_STATE_T = 0, ST_STATE_LAMBDA = 1, ST_STATE_RHS = 2, ST_STATE_ADJ_RHS = 3 };
enum { ST_COARSEN_SEMI = 0, ST_COARSEN_FULL = 1 };
/* Coarsest-level solver: AUTO = dense FP64 inverse when the coarsest level has at most 4096
 * nodes, else Jacobi-GMRES; DENSE = always the dense inverse (error above 4096 nodes);
 * GMRES = FP64 right-Jacobi-preconditioned restarted GMRES(16), the paper's coarsest solve
 * (Sec. 3.2), stopped at coarse_rtol or after coarse_max_it iterations. */
enum { ST_COARSE_AUTO = 0, ST_COARSE_DENSE = 1, ST_COARSE_GMRES = 2 };
/* Multigrid smoother of the levels above the coarsest (st_mesh_desc.smoother). */
enum { ST_SMOOTH_GMRES = 0, ST_SMOOTH_JACOBI = 1 };

/* Modified SIMP (Sec. 2.2): C = C_ins + (C_con - C_ins) g^p_c, k = k_ins + (k_con - k_ins) g^p_k.
 * Integer powers p_c, p_k >= 1. */
typedef struct {
    double C_ins, C_con, k_ins, k_con;
    int p_c, p_k;
} st_material;

/* Mesh and hierarchy description (Sec. 3.1.2 mesh, Algorithm 1 coarsening). */
typedef struct {
    int ndim_space;          /* 2 or 3 spatial dimensions */
    int n[3];                /* spatial element counts (x, y, z); n[2] ignored in 2D */
    int n_t;                 /* time element count */
    double ext[3];           /* spatial extents; element size h_d = ext[d] / n[d] */
    double tau;              /* final time (rescaled, Sec. 2.1) */
    st_material mat;
    int bc;                  /* ST_BC_*: sink patch on x=0 (LEFT) or y=0 (BOTTOM), all walls, none.
                                T = 0 on the t = 0 plane always (initial condition). */
    double bc_width;         /* patch width as a fraction of the edge length (paper: 0.1) */
    double lambda_crit;      /* Algorithm 1 threshold (paper: 0.5) */
    long long coarse_dof_cap;/* coarsen until a level has at most this many nodes (<= 4096) */
    int max_levels;          /* 0 = no limit */
    int coarsening;          /* ST_COARSEN_SEMI (Algorithm 1) or ST_COARSEN_FULL (ablation) */
    int device;              /* CUDA device ordinal */
    int coarse_solver;       /* ST_COARSE_* */
    int coarse_max_it;       /* Jacobi-GMRES iterations on the coarsest level (0: 200) */
    double coarse_rtol;      /* its relative residual target (0: 1e-6) */
    int march_blocks;        /* tuning: thread-block budget of the time-marching stencil kernels
                                (0: 912, two waves on 152 SMs; at most 4096); a smaller budget
                                gives each block a longer time chunk */
    int smoother;            /* ST_SMOOTH_GMRES: the paper's Jacobi-GMRES; ST_SMOOTH_JACOBI: damped
                                Jacobi sweeps x += omega D^-1 (b - J x), a cheaper variant (the
                                paper's outlook); st_options.smooth_steps counts sweeps */
    double smoother_omega;   /* Jacobi damping omega in (0, 1] (default 0.5; 0.7 lets the V-cycle
                                diverge on some space-time designs) */
} st_mesh_desc;

typedef struct {
    int kind;                /* ST_SRC_UNIFORM: Q = q0; ST_SRC_SIN_T: Q = q0 (a + b sin(2 pi f t));
                                ST_SRC_GAUSSIAN (Example 2, Sec. 2.3.2; 2 space dimensions only):
                                Q = q0 exp(-|x - c(t)|^2 / (2 a^2)), c(t) = centre of the domain
                                + b (cos(f t + pi/2), sin(f t + pi/2)): width a > 0, radius b,
                                angular frequency f.  Every kind is integrated by 2-point Gauss
                                per axis and element. */
    double q0, a, b, f;
} st_source;

typedef struct {
    double rtol;             /* stop when ||f - J s||_2 <= rtol ||f||_2 (true residual) */
    int max_it;              /* cap on outer iterations (all restarts together) */
    int restart;             /* FGMRES restart length m (<= 32) */
    int precision;           /* ST_PREC_MIXED: FP32 multigrid, or ST_PREC_FP64 */
    int warm_start;          /* 1: start from the stored state (Sec. 3.2 warm start) */
    int smooth_steps;        /* Jacobi-GMRES smoothing iterations per pre/post step (<= 16) */
    int use_graphs;          /* 1: replay the V-cycle as a captured CUDA graph */
} st_options;

typedef struct {
    int kind;                /* ST_OBJ_COMPLIANCE: phi = f^T s; ST_OBJ_PNORM: Sec. 3.3.1 p-norm */
    int P;                   /* p-norm exponent (paper: 20) */
} st_objective;

typedef struct {
    int outer_its;           /* FGMRES iterations (= V-cycles applied) */
    int restarts;
    int converged;
    double rel_res;          /* true ||f - J s|| / ||f|| at exit */
    double rel_res_est;      /* FGMRES estimate at exit */
    double seconds;          /* wall time of the call */
    double norm_f;
} st_stats;

typedef struct {
    int n_levels;
    long long n_nodes;       /* fine-level DOFs (Dirichlet nodes included) */
    long long n_elem;
    long long device_bytes;  /* device memory currently held by the mesh */
} st_mesh_info;

typedef struct {
    int n[3];
    int n_t;
    long long n_nodes;
    int to_next;             /* 0 space, 1 time, 2 full, -1 coarsest */
    double h[3], dt;
} st_level_info;

typedef struct st_mesh st_mesh;

const char* st_version(void);
const char* st_last_error(void);
void st_mesh_desc_default(st_mesh_desc* d);
void st_options_default(st_options* o);

/* Host-only: the multigrid hierarchy Algorithm 1 gives for d (no device work).  Writes up to
 * max_out levels to out (finest first) and the level count to *n_levels. */
st_status st_plan_hierarchy(const st_mesh_desc* d, st_level_info* out, int max_out, int* n_levels);

/* Create a mesh: validates d, builds the hierarchy by Algorithm 1 (host) and
 * allocates its device memory.  *out receives the handle. */
st_status st_create_mesh(const st_mesh_desc* d, st_mesh** out);
st_status st_destroy_mesh(st_mesh* m);
st_status st_mesh_info_get(const st_mesh* m, st_mesh_info* info);
st_status st_level_info_get(const st_mesh* m, int level, st_level_info* info);
/* Queue the mesh's work on `stream` (a cudaStream_t; NULL = the mesh's own stream). */
st_status st_set_stream(st_mesh* m, void* stream);
st_status st_synchronize(st_mesh* m);

/* Set the density design (Sec. 2.2.1).  layout ST_DESIGN_EXTRUDED: count = nx*ny(*nz),
 * constant along time (Sec. 3.4.1); ST_DESIGN_SPACETIME: count = number of elements.
 * Values are clipped to [0, 1]; a NaN or infinite value returns ST_ERR_NUMERIC and leaves the
 * mesh without a design (solves return ST_ERR_STATE until a valid design is set).  Builds the Galerkin coarse operators (J_{l+1} = P^T J_l P,
 * Sec. 3.2), the 27-point stencils of time-constant 2-D designs and, for the dense coarsest
 * solve, the inverse of the coarsest operator; the Jacobi diagonals follow at the next solve. */
st_status st_set_design(st_mesh* m, const double* gamma, int layout, size_t count, int mem);

/* Forward solve J s = f (Sec. 3.1.2) with f from `q` (2-point Gauss in time per element).
 * ST_ERR_NOT_CONVERGED keeps the best iterate and fills stats.  Non-finite source parameters
 * return ST_ERR_ARG; a NaN or Inf that reaches the residual (for example from a warm-start
 * state) returns ST_ERR_NUMERIC.  ST_ERR_TIMEOUT: a bounded grid-barrier wait of the opt-in
 * persistent coarse V-cycle tail gave up (the result is then not to be trusted). */
st_status st_solve_forward(st_mesh* m, const st_source* q, const st_options* o, st_stats* stats);

/* Objective phi (*phi_out) from the stored state and the adjoint solve J^T Lambda =
 * (d phi / d s)^T (Sec. 3.3.3), Lambda = 0 at prescribed nodes.  Needs a forward solve. */
st_status st_solve_adjoint(st_mesh* m, const st_objective* obj, const st_options* o,
                           double* phi_out, st_stats* stats);

/* PDE filter of an element field (Sec. 3.3.2): solves -div(D grad psi) + psi = gamma over the
 * space-time domain, D = diag(r_x^2/12 per spatial axis, r_t^2/12 in time), natural boundary
 * conditions, with the mesh's trilinear space-time elements ((M + K) psi = T gamma, T_ie =
 * v_e / n_v) by Jacobi-preconditioned conjugate gradients to ||r|| <= rtol ||T gamma||, and
 * returns the element means of psi.  in/out: element fields of `count` values (spatial elements
 * for a time-constant field, solved on one slab, or all space-time elements), host or device
 * per mem.  r_x, r_t <= 0 take the paper's minimum 2.4 h_min and 2.4 dt.  The filtered field
 * of a field equal to 1 is 1 and the element sum is preserved.  The filter is symmetric, so the
 * chain rule of the sensitivities is the same call: d phi / d gamma = filter(H'(gamma~) *
 * d phi / d gamma_bar).  *iterations (may be NULL) receives the CG iterations.
 * ST_ERR_NOT_CONVERGED: max_it reached (out holds the last iterate's means); ST_ERR_NUMERIC:
 * a NaN or infinite input.  Uses scratch memory held by the mesh (allocated at the first call). */
st_status st_filter(st_mesh* m, const double* in, double* out, size_t count, int mem, double r_x, double r_t,
                    double rtol, int max_it, int* iterations);
/* Heaviside projection of Sec. 3.3.2, element by element on the mesh's device:
 * out = (tanh(beta eta) + tanh(beta (in - eta))) / (tanh(beta eta) + tanh(beta (1 - eta))) and its
 * derivative dout (either may be NULL).  Paper values: eta = 0.5, beta = 32. */
st_status st_heaviside(st_mesh* m, const double* in, double* out, double* dout, size_t count, int mem, double beta,
                       double eta);

/* Batched solves (no counterpart in the paper: concurrent design iterations of the paper's
 * optimisation loop issue many such solves).  The meshes (all on one device, each at most
 * once) are solved together: every FGMRES restart cycle of every mesh is captured into ONE CUDA
 * graph, in which the outer iterations run inside conditional graph nodes (a WHILE node over the
 * iterations, a SWITCH over the iteration index) and the convergence test and the stop decision
 * are taken on the device; one graph launch advances all meshes by a whole restart cycle and the
 * host synchronises once per cycle, not once per iteration.  Results are bit-identical to
 * st_solve_forward / st_solve_adjoint of each mesh alone.  The graph runs on the first mesh's
 * stream.  q, obj, phi_out, stats and status are arrays of `count` entries (stats, status and
 * phi_out may be NULL); status[k] is mesh k's outcome (ST_OK, ST_ERR_NOT_CONVERGED,
 * ST_ERR_NUMERIC).  Returns ST_OK when every mesh succeeded, else the first failure; argument
 * and call-order errors (ST_ERR_ARG, ST_ERR_STATE) leave every mesh untouched.
 * All meshes use the same options o (NULL: defaults). */
st_status st_solve_forward_batch(st_mesh* const* m, int count, const st_source* q, const st_options* o,
                                 st_stats* stats, st_status* status);
st_status st_solve_adjoint_batch(st_mesh* const* m, int count, const st_objective* obj, const st_options* o,
                                 double* phi_out, st_stats* stats, st_status* status);

/* Sensitivities d phi / d gamma_e = -Lambda_e^T (dJ_e / d gamma_e) s_e (Sec. 3.3.3); for
 * an extruded design summed over time (transpose of the extrusion, Sec. 3.4.1).
 * count must equal the design size. */
st_status st_sensitivities(st_mesh* m, double* out, size_t count, int mem);

/* Copy a stored node vector (ST_STATE_*) to `out` (count = fine DOFs). */
st_status st_get_state(st_mesh* m, int which, double* out, size_t count, int mem);
/* Overwrite the stored state s (e.g. an initial guess for a warm start). */
st_status st_set_state(st_mesh* m, const double* s, size_t count, int mem);

/* ---- Component entry points (used by the parity tests; same kernels as the solve) ----
 * precision selects the multigrid copy: ST_PREC_MIXED -> float vectors (level 0 applies with
 * FP32 stencils built from the FP64 design on time-constant 2-D designs, else with the BF16
 * design), ST_PREC_FP64 -> double vectors.  level 0 with precision
 * ST_PREC_FP64 is also the FP64 operator of the outer Krylov solver.  All vectors are
 * device pointers of the level's node count. */
st_status st_op_apply(st_mesh* m, int level, int precision, int transpose, const void* x, void* y);
st_status st_op_diag(st_mesh* m, int level, int precision, void* d);
/* r_c = P^T r_f (masked), from `level` to level + 1. */
st_status st_restrict(st_mesh* m, int level, int precision, const void* r_f, void* r_c);
/* x_f += P x_c (masked), from level + 1 to `level`. */
st_status st_prolong(st_mesh* m, int level, int precision, const void* x_c, void* x_f);
/* x <- `steps` Jacobi-GMRES iterations on A_level x = b starting from x (zero_init: from 0). */
st_status st_smooth(st_mesh* m, int level, int precision, int transpose, const void* b, void* x,
                    int steps, int zero_init);
/* x = V-cycle(b) on level 0, i.e. one application of the preconditioner. */
st_status st_vcycle(st_mesh* m, int precision, int transpose, const void* b, void* x);
/* Export level `level` (>= 1) element matrices in FP64 block form: for each stored element,
 * 4 blocks (a_t, b_t) in order 00, 01, 10, 11 of the packed upper triangle of the symmetric
 * spatial block (row-major, i <= j).  Extruded designs store 2 versions (first slab, other
 * slabs) per spatial element.  count is in doubles; host pointer. */
st_status st_level_elements(st_mesh* m, int level, double* out, size_t count);
/* Copy the FP64 inverse of the coarsest operator (n x n, row-major) to a host buffer.
 * ST_ERR_STATE when the coarsest level is solved by Jacobi-GMRES (no dense inverse). */
st_status st_coarse_inverse(st_mesh* m, double* out, size_t count);

/* ---- Diagnostics (no counterpart in the paper) ----
 * CUDA-event timing of the level-0 smoother operator apply (w = A D^-1 u_j, the most
 * frequently launched stencil kernel of the V-cycle, Sec. 3.2) inside real solves.
 * enable = 1 resets the totals and records an event pair around every such launch on the
 * mesh stream (event nodes inside captured V-cycles; cached V-cycle graphs are rebuilt when
 * the setting changes); the pairs are read after the host synchronisation that ends each
 * outer Krylov iteration.  enable = 0 stops recording and keeps the totals.  Synchronises
 * the mesh stream.  Errors: ST_ERR_ARG (null mesh), ST_ERR_CUDA (event creation). */
st_status st_apply_timer(st_mesh* m, int enable);
/* Totals since the last st_apply_timer(m, 1): summed launch time in ms and launch count. */
st_status st_apply_timer_read(st_mesh* m, double* total_ms, long long* launches);

/* ---- Serving: continuous batching of forward + adjoint + sensitivity requests ---- */
typedef struct {
    st_mesh_desc mesh;
    const double* gamma;     /* host design, copied at submit */
    int layout;
    size_t count;
    st_source source;
    st_objective objective;
    st_options options;
    int want_gradient;       /* 1: keep the sensitivities for st_poll */
} st_request;

typedef struct {
    st_status status;
    double phi;
    st_stats forward, adjoint;
    double latency_s;        /* submit -> completion */
    double queue_s;          /* submit -> admission */
    long long footprint;     /* admitted device bytes */
    int batch;               /* requests solved together with this one in shared graph launches
                                (1: alone) */
} st_result;

typedef struct {
    long long hbm_budget;    /* device bytes the server may hold for requests */
    int max_inflight;        /* concurrent slots, each solving one batch at a time */
    int device;
    int max_batch;           /* requests a slot may solve together in one batch (0: 8; 1: no batching) */
    long long batch_nodes;   /* only requests of at most this many nodes share a batch (0: 2^21) */
} st_server_desc;

typedef struct st_server st_server;

st_status st_server_create(const st_server_desc* d, st_server** out);
/* Waits for in-flight requests, then releases everything. */
st_status st_server_destroy(st_server* s);
/* Queue a request; *ticket identifies it.  ST_ERR_BUSY if its footprint can never fit. */
st_status st_submit(st_server* s, const st_request* r, uint64_t* ticket);
/* *done = 1 once finished; out filled then.  grad (host, may be NULL) receives the
 * sensitivities if requested (count = design size).  A finished ticket is released by the
 * first st_poll that returns done = 1. */
st_status st_poll(st_server* s, uint64_t ticket, st_result* out, double* grad, size_t count, int* done);
/* Cancel a request that is still queued (not yet admitted to a slot).  Returns ST_OK and
 * marks it finished with result status ST_ERR_CANCELLED (release it with st_poll as usual);
 * ST_ERR_BUSY if it is already running on the device (it then runs to completion),
 * ST_ERR_STATE if it has finished, ST_ERR_NOT_FOUND for an unknown or released ticket. */
st_status st_cancel(st_server* s, uint64_t ticket);
/* Number of kernels this library has launched in the process so far (kernels inside
 * replayed CUDA graphs included); a diagnostic for benchmarks. */
long long st_kernel_launches(void);

/* Diagnostic (no counterpart in the paper): measured FP64 FMA throughput of `device` in
 * TFLOP/s (2 flops per FMA), from a kernel of independent FMA chains on every SM, best of 5
 * CUDA-event-timed runs.  It is the denominator of the roofline of the FP64 operator applies
 * of the outer Krylov solver.  Allocates and frees a small scratch buffer. */
st_status st_fp64_fma_rate(int device, double* tflops);

/* Device-memory estimate used by admission control for a mesh description. */
long long st_footprint_bytes(const st_mesh_desc* d, int precision, int restart);

/* ---- Method of Moving Asymptotes with one constraint (Sec. 3.3.3) ----
 * The optimiser of the topology-optimisation loop: min f0(x) s.t. g1(x) <= 0, x_min <= x <= x_max
 * (the paper's volume constraint), Svanberg's method with the asymptote rule, move limits and
 * convex approximations below, the subproblem solved through its one-multiplier dual.  The
 * paper cites a modified form of Guest et al.'s initial asymptotes without values; s0 is that
 * reading.  Parameters (st_mma_params_default): first two iterations' asymptotes at
 * x -/+ s0 (x_max - x_min) (0.05); later ones moved by incr (1.2) where the last two steps kept
 * their sign and decr (0.7) where it flipped; move limit `move` (0.2) of the span; regularisation
 * raa (1e-5) of the approximation terms; multiplier cap lam_max (1e40), reached only when the
 * approximated constraint cannot be met within the move limits (the step then goes to its most
 * feasible point). */
typedef struct {
    double s0, incr, decr, move, raa, lam_max;
} st_mma_params;
typedef struct st_mma st_mma;

void st_mma_params_default(st_mma_params* p);
/* Device state for n variables on the current device (previous two iterates, asymptotes,
 * subproblem terms: 10 n doubles).  p NULL: the defaults.  ST_ERR_ARG for n < 1 or parameters
 * outside (s0 > 0, incr >= 1, 0 < decr <= 1, move > 0, raa > 0, lam_max > 1, all finite); ST_ERR_OOM. */
st_status st_mma_create(long long n, const st_mma_params* p, st_mma** out);
st_status st_mma_destroy(st_mma* h);
/* One MMA iteration it (1, 2, 3, ... in order; the asymptote rule uses the two previous
 * iterates the object keeps) on `stream`: x (device, n doubles) is replaced by the new iterate;
 * df0 and dg1 (device, n doubles) are the gradients of the objective and the constraint at x,
 * g1 the constraint's value there.  The multiplier goes to *lam (may be NULL).  The dual's
 * bisection reads one partial sum per trial from the device, so the call returns after the
 * update has completed.  ST_ERR_ARG for null pointers, it < 1, x_max <= x_min or a non-finite g1. */
st_status st_mma_update(st_mma* h, int it, double* x, const double* df0, double g1, const double* dg1, double xmin,
                        double xmax, void* stream, double* lam);

/* ---- Topology-optimisation loop (Sec. 3.3, the nested formulation of the optimisation
 * problem): one design iteration per st_topopt_step, every step on the mesh's device and stream:
 *   gamma~ = F gamma (PDE filter, Sec. 3.3.2), gamma_bar = H(gamma~) (projection),
 *   st_set_design(gamma_bar), forward solve, objective phi and adjoint solve, d phi / d gamma_bar,
 *   chain rule d phi / d gamma = F (H'(gamma~) d phi / d gamma_bar) (F symmetric: uniform
 *   elements), the volume constraint chi = sum gamma_bar_e v_e / (v_f |Pi|) - 1 on the physical
 *   design with d chi / d gamma = F (H'(gamma~) / (v_f N_e)) (Sec. 3.3.3), and one MMA update of
 *   gamma in [0, 1] (st_mma_update).  The objective enters MMA scaled by obj_scale / phi_1, phi_1
 *   its value at the first iteration.  From the second iteration on the forward and adjoint
 *   solves start from the previous design's solutions when warm_start is set (Sec. 3.2). */
typedef struct {
    double vf;          /* volume fraction v_f, 0 < vf < 1 (paper: 0.3) */
    double r_x, r_t;    /* filter radii; <= 0 selects the minimum 2.4 h and 2.4 dt */
    double beta, eta;   /* projection sharpness and threshold (paper: 32, 0.5) */
    int objective;      /* ST_OBJ_PNORM (paper, P = 20) or ST_OBJ_COMPLIANCE */
    int P;              /* p-norm exponent */
    double obj_scale;   /* MMA sees obj_scale * phi / phi_1 (default 10) */
    double filter_rtol; /* filter CG tolerance (default 1e-10) */
    int filter_max_it;  /* filter CG iteration cap (default 2000) */
    int warm_start;     /* 1: warm-started solves from the second iteration (default 1) */
    st_mma_params mma;  /* optimiser parameters (st_mma_params_default) */
} st_topopt_params;
typedef struct {
    int iteration;      /* design iterations taken, this one included */
    double phi;         /* objective at the design entering this iteration (unscaled) */
    double chi;         /* volume constraint at that design (<= 0: satisfied) */
    double lam;         /* MMA multiplier of the volume constraint */
    double change;      /* max_e |gamma_e after - gamma_e before| */
    st_stats forward;   /* the forward solve */
    st_stats adjoint;   /* the adjoint solve */
    int filter_its;     /* CG iterations of the three filter solves together */
    double seconds;     /* host wall time of the iteration */
    double filter_seconds;  /* of which: the three filter solves */
    double design_seconds;  /* projection and st_set_design */
    double mma_seconds;     /* volume sum and the MMA update */
} st_topopt_stats;
typedef struct st_topopt st_topopt;
enum { ST_TO_GAMMA = 0, ST_TO_GAMMA_TILDE = 1, ST_TO_GAMMA_BAR = 2, ST_TO_DPHI = 3, ST_TO_DCHI = 4 };

void st_topopt_params_default(st_topopt_params* p);
/* An optimisation of mesh m (which must outlive the handle) from the initial design gamma0
 * (count values, layout ST_DESIGN_*, host or device per mem; clipped to [0, 1]).  The handle
 * owns 8 count doubles of device memory plus an st_mma.  ST_ERR_ARG: count does not match the
 * layout, vf outside (0, 1), beta <= 0, eta outside (0, 1), obj_scale <= 0, an unknown
 * objective or P outside [1, 64]; ST_ERR_NUMERIC: a non-finite gamma0; ST_ERR_OOM. */
st_status st_topopt_create(st_mesh* m, const st_topopt_params* p, const double* gamma0, int layout, size_t count,
                           int mem, st_topopt** out);
st_status st_topopt_destroy(st_topopt* h);
/* One design iteration with source q and solver options o (NULL: defaults; o->warm_start is
 * replaced by the handle's rule).  On return the handle holds the new design; stats (may be
 * NULL) describe the iteration.  ST_ERR_NOT_CONVERGED: a solve or a filter stopped at its
 * iteration cap; the iteration was still completed from its last iterate.  Other errors leave
 * the design unchanged. */
st_status st_topopt_step(st_topopt* h, const st_source* q, const st_options* o, st_topopt_stats* stats);
/* Copy one field (ST_TO_*, count values: gamma, gamma~, gamma_bar, and the chain-ruled
 * gradients d phi / d gamma and d chi / d gamma of the last iteration, the first scaled as MMA
 * saw it) to out (host or device per mem).  ST_ERR_STATE for the fields an iteration makes
 * before the first st_topopt_step. */
st_status st_topopt_get(st_topopt* h, int which, double* out, size_t count, int mem);

/* ---- Reference time stepping (Sec. 4): the comparison solver of the paper, first-order
 * backward differences (BDF1) on the spatial mesh with consistent capacity-weighted mass,
 *   (M_C + dt K_k) T^{n+1} = M_C T^n + dt F(t_{n+1}),  T^0 = 0,  dt = tau / n_t,
 * step n taking the design of slab n and F_i(t) = Q(t) int N_i (uniform and sine sources), the
 * spatial sink prescribed at every step.  Each step is one FGMRES solve preconditioned by the
 * library's multigrid on a one-slab mesh whose upper-plane block is exactly M_C + dt K_k
 * (conductivities tripled, final time dt): Algorithm 1 coarsens it in space only, the paper's
 * spatial multigrid for time stepping.  Each solve starts from the previous plane. */
typedef struct {
    int steps;              /* steps taken */
    long long outer_its;    /* FGMRES iterations of all steps */
    int max_outer_its;      /* of the worst step */
    double max_rel_res;     /* largest true relative residual at a step's exit */
    double seconds;         /* host wall time of the call */
} st_bdf1_stats;
typedef struct st_bdf1 st_bdf1;
/* The solver for the space-time problem d (its n_t steps, tau, material, sink, hierarchy
 * options; the step mesh copies d with n_t = 1).  Holds the step mesh, the design and the
 * trajectory ((n_t + 1) planes) on the device.  Errors as st_create_mesh; ST_ERR_OOM. */
st_status st_bdf1_create(const st_mesh_desc* d, st_bdf1** out);
st_status st_bdf1_destroy(st_bdf1* h);
/* The design (layout ST_DESIGN_*, count values, host or device per mem; clipped to [0, 1]).
 * ST_ERR_NUMERIC for a NaN or infinite value in the first slab (later slabs are checked at
 * their step). */
st_status st_bdf1_set_design(st_bdf1* h, const double* gamma, int layout, size_t count, int mem);
/* Run the n_t steps with source q (ST_SRC_UNIFORM or ST_SRC_SIN_T; others ST_ERR_ARG) and the
 * step solves' options o (NULL: defaults; warm_start is always on).  T (may be NULL; host or
 * device per mem) receives the trajectory, count = (n_t + 1) * nodes per plane, plane n at
 * t = n dt.  ST_ERR_NOT_CONVERGED: a step stopped at max_it (the trajectory is complete). */
st_status st_bdf1_forward(st_bdf1* h, const st_source* q, const st_options* o, double* T, size_t count, int mem,
                          st_bdf1_stats* stats);
/* Discrete adjoint of the stepping for the p-norm objective of Sec. 3.3.1 (exponent P in [1, 64])
 * over the space-time elements of the last forward trajectory: from the last step backwards
 *   A_{m-1} Lambda^m = d phi / d T^m + M_m Lambda^{m+1},  Lambda^{n_t + 1} = 0,
 * (A_n = M_C + dt K_k and M_n = M_C of slab n), each solve started from Lambda^{m+1}.  *phi
 * (may be NULL) receives the objective; Lambda (may be NULL; host or device per mem, count =
 * (n_t + 1) plane nodes) the multipliers, plane 0 zero.  ST_ERR_STATE without a forward run. */
st_status st_bdf1_adjoint(st_bdf1* h, int P, const st_options* o, double* phi, double* Lambda, size_t count, int mem,
                          st_bdf1_stats* stats);
/* d phi / d gamma_e = -Lambda^{n+1}_e . (C'_e M_e (T^{n+1} - T^n)_e + dt k'_e K_e T^{n+1}_e) for
 * element e of slab n, summed over the slabs for an extruded design; count = the design size.
 * ST_ERR_STATE without an adjoint run. */
st_status st_bdf1_sensitivities(st_bdf1* h, double* out, size_t count, int mem);

/* ---- Allocation-free residual for callers that cannot allocate device memory ----
 * The paper has no counterpart; this entry point exists for callers that must not call
 * cudaMalloc (code running inside another framework's stream capture or memory pool, or
 * a real-time loop).  It computes r = f - J x and ||r||_2 for the FP64 fine-level operator
 * of mesh description d and design gamma (layout ST_DESIGN_*; values used as given, not
 * clipped), matrix free, queued on
 * `stream` (a cudaStream_t, NULL = legacy default stream).  All pointers are device
 * pointers owned by the caller: gamma (design size), x, f, r (node count each) and norm
 * (one double, written when the stream reaches the kernel).  No mesh is needed and nothing
 * is allocated: the only scratch is a static 32 KiB device array that every GPU loading
 * the library keeps until exit.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress), so make it before any stream capture; after it, a call can be
 * captured into a CUDA graph and replayed.  The address is kept per device for the process,
 * so a cudaDeviceReset of that device is not supported afterwards.  Limits: the x-y plane may
 * hold at most 4096 tiles of 32 x 8 nodes (e.g. 1024 x 1024 spatial elements) and the
 * mesh at most 2^31 - 1 nodes; larger sizes return ST_ERR_ARG.  All calls share the one
 * array (it keeps the last call's partial sums; the completion counter is cleared at the
 * start of each call), so calls that overlap on the GPU (different streams, or host
 * threads on the same device) race and must be serialised by the caller. */
st_status st_residual_norm_noalloc(const st_mesh_desc* d, const double* gamma, int layout, const double* x,
                                   const double* f, double* r, double* norm, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ST_H */
