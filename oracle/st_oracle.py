"""FP64 CPU oracle for the space-time FE heat-conduction solve (arXiv 2508.09589).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this module.  The product path (the CUDA
library and its Python binding) never calls it and shares no code with it.

Everything here is plain and slow on purpose: element integrals by Gauss
quadrature of the weak form, global assembly into a scipy sparse matrix, a
direct sparse solve, and sparse matrix products for the multigrid transfer
and Galerkin operators.  Each function names the passage of the paper it
follows.  Readings of points the paper leaves open are marked "Reading".

Notation follows the paper: s (state, nodal temperatures), J (system matrix),
f (source vector), Lambda (adjoint), gamma (design), C and k (capacity and
conductivity by modified SIMP), tau (final time), Delta x, Delta t.

Node numbering: C order over (t, [z,] y, x) with x fastest and time slowest.
Element numbering: C order over (slab, [z,] y, x).  Local element node a has
bits (a_t, [a_z,] a_y, a_x) with a_x the lowest bit.

Parity status: every function below is pinned by a CPU test (tests/test_oracle_*.py);
none is "parity unpinned".
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# Material interpolation (Sec. 2.2, modified SIMP equations)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Material:
    C_ins: float = 0.5
    C_con: float = 1.0
    k_ins: float = 0.03
    k_con: float = 3.0
    p_c: int = 2
    p_k: int = 3


def simp_C(m: Material, g):
    """C(gamma) = C_ins + (C_con - C_ins) gamma^p_c."""
    return m.C_ins + (m.C_con - m.C_ins) * g ** m.p_c


def simp_k(m: Material, g):
    """k(gamma) = k_ins + (k_con - k_ins) gamma^p_k."""
    return m.k_ins + (m.k_con - m.k_ins) * g ** m.p_k


def simp_dC(m: Material, g):
    """dC/dgamma."""
    return m.p_c * (m.C_con - m.C_ins) * g ** (m.p_c - 1)


def simp_dk(m: Material, g):
    """dk/dgamma."""
    return m.p_k * (m.k_con - m.k_ins) * g ** (m.p_k - 1)


# ----------------------------------------------------------------------------
# Mesh (Sec. 3.1.2: regular cuboid mesh of trilinear space-time elements)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Mesh:
    ns: Tuple[int, ...]                 # spatial element counts, x first
    nt: int                             # time element count
    ext: Tuple[float, ...] = ()         # spatial extents (default unit length per axis)
    tau: float = 1.0                    # final time
    mat: Material = Material()
    bc: str = "patch_left"              # patch_left | patch_bottom | all_walls | none
    bc_width: float = 0.1               # patch width as a fraction of the edge length

    def __post_init__(self):
        if not self.ext:
            object.__setattr__(self, "ext", tuple(1.0 for _ in self.ns))

    @property
    def sd(self) -> int:
        return len(self.ns)

    @property
    def h(self) -> Tuple[float, ...]:
        return tuple(e / n for e, n in zip(self.ext, self.ns))

    @property
    def dt(self) -> float:
        return self.tau / self.nt

    @property
    def node_shape(self) -> Tuple[int, ...]:
        return (self.nt + 1,) + tuple(n + 1 for n in reversed(self.ns))

    @property
    def elem_shape(self) -> Tuple[int, ...]:
        return (self.nt,) + tuple(reversed(self.ns))

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.node_shape))

    @property
    def n_elem(self) -> int:
        return int(np.prod(self.elem_shape))

    @property
    def nv(self) -> int:
        return 2 ** (self.sd + 1)


def with_size(m: Mesh, ns: Sequence[int], nt: int, tau: Optional[float] = None) -> Mesh:
    return Mesh(tuple(ns), nt, m.ext, m.tau if tau is None else tau, m.mat, m.bc, m.bc_width)


def element_connectivity(m: Mesh) -> np.ndarray:
    """conn[e, a] = global node of local node a of element e."""
    shape = m.node_shape
    strides = np.cumprod((1,) + tuple(reversed(shape[1:])))[::-1]  # C-order strides
    eidx = np.indices(m.elem_shape).reshape(len(shape), -1)  # (axis, e)
    conn = np.zeros((m.n_elem, m.nv), dtype=np.int64)
    for a in range(m.nv):
        # bit d of a (d = 0 is x) -> offset along spatial axis d; top bit -> time
        off = [0] * len(shape)
        off[0] = (a >> m.sd) & 1
        for d in range(m.sd):
            off[len(shape) - 1 - d] = (a >> d) & 1
        idx = sum((eidx[ax] + off[ax]) * strides[ax] for ax in range(len(shape)))
        conn[:, a] = idx
    return conn


def node_coords(m: Mesh) -> List[np.ndarray]:
    """[t, (z,) y, x] coordinates of every node, each flattened in node order."""
    grids = [np.arange(m.nt + 1) * m.dt] + [np.arange(n + 1) * hh for n, hh in
                                              zip(reversed(m.ns), reversed(m.h))]
    mesh = np.meshgrid(*grids, indexing="ij")
    return [g.reshape(-1) for g in mesh]


# ----------------------------------------------------------------------------
# Dirichlet set.  Reading: T = 0 on the whole t = 0 plane (initial condition),
# plus the spatial sink, applied at every time.  A patch of relative width w
# centred on an edge (or face) contains node j of an axis with n elements iff
# |2 j - n| <= w n (+1e-9), i.e. |x_j - L/2| <= w L / 2.
# ----------------------------------------------------------------------------
def _patch_mask_1d(n: int, width: float) -> np.ndarray:
    j = np.arange(n + 1)
    return np.abs(2 * j - n) <= width * n + 1e-9


def dirichlet_mask(m: Mesh) -> np.ndarray:
    """Boolean node mask, True where T is prescribed (= 0)."""
    shape = m.node_shape
    D = np.zeros(shape, dtype=bool)
    D[0] = True  # t = 0 plane
    sd = m.sd
    # spatial axes in array order: axis 1 + (sd-1-d) holds spatial direction d
    ax = lambda d: 1 + (sd - 1 - d)
    if m.bc == "none":
        pass
    elif m.bc == "all_walls":
        for d in range(sd):
            sl = [slice(None)] * len(shape)
            sl[ax(d)] = 0
            D[tuple(sl)] = True
            sl[ax(d)] = -1
            D[tuple(sl)] = True
    elif m.bc in ("patch_left", "patch_bottom"):
        face_dir = 0 if m.bc == "patch_left" else 1
        sel = np.ones(shape[1:], dtype=bool)
        for d in range(sd):
            a = ax(d) - 1
            bshape = [1] * sd
            bshape[a] = m.ns[d] + 1
            if d == face_dir:
                v = np.zeros(m.ns[d] + 1, dtype=bool)
                v[0] = True
            else:
                v = _patch_mask_1d(m.ns[d], m.bc_width)
            sel = sel & v.reshape(bshape)
        D[:] |= sel[None]
    else:
        raise ValueError(m.bc)
    return D.reshape(-1)


# ----------------------------------------------------------------------------
# Element matrices (Sec. 3.1.1 weak form with time artificial diffusion
# k_ad = C dt / 2) by Gauss quadrature on one Delta x ... x Delta t brick.
# ----------------------------------------------------------------------------
def gauss_1d(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre points and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _basis_1d(xi):
    """Linear 1D shape functions and derivatives on [0,1]: phi_0 = 1 - xi, phi_1 = xi."""
    return (np.array([1.0 - xi, xi]), np.array([-1.0, 1.0]))


def element_matrices(h: Sequence[float], dt: float, ngauss: int = 3):
    """Unit-coefficient element matrices of the weak form.

    Jc[a, b] = int N_a dN_b/dt + (dt/2) dN_a/dt dN_b/dt  (capacity part, C = 1,
               including the stabilising time diffusion k_ad = C dt / 2)
    Jk[a, b] = int sum_d dN_a/dx_d dN_b/dx_d             (conductivity part, k = 1)
    Row index a is the test function, column b the trial function.
    """
    sd = len(h)
    nv = 2 ** (sd + 1)
    gp, gw = gauss_1d(ngauss)
    sizes = list(h) + [dt]  # physical size per local axis: x, y, (z), t
    Jc = np.zeros((nv, nv))
    Jk = np.zeros((nv, nv))
    for q in itertools.product(range(ngauss), repeat=sd + 1):
        # q[d] for spatial d, q[sd] for time
        wq = np.prod([gw[qi] * sizes[d] for d, qi in enumerate(q)])
        N = np.ones(nv)
        dN = np.ones((sd + 1, nv))  # physical derivatives
        for a in range(nv):
            for d in range(sd + 1):
                bit = (a >> d) & 1
                phi, dphi = _basis_1d(gp[q[d]])
                N[a] *= phi[bit]
                for dd in range(sd + 1):
                    dN[dd, a] *= (dphi[bit] / sizes[d]) if dd == d else phi[bit]
        dNt = dN[sd]
        Jc += wq * (np.outer(N, dNt) + 0.5 * dt * np.outer(dNt, dNt))
        for d in range(sd):
            Jk += wq * np.outer(dN[d], dN[d])
    return Jc, Jk


# ----------------------------------------------------------------------------
# Design -> per-element coefficients (Sec. 2.2.1: extruded or space-time design)
# ----------------------------------------------------------------------------
def element_gamma(m: Mesh, gamma: np.ndarray) -> np.ndarray:
    """Per-element design, flattened in element order.  A design with the spatial
    shape only is extruded along time (Sec. 3.4.1); a full shape is a space-time design."""
    g = np.asarray(gamma)
    sp_shape = tuple(reversed(m.ns))
    if g.shape == sp_shape or g.size == int(np.prod(sp_shape)):
        g = np.broadcast_to(g.reshape(sp_shape)[None], m.elem_shape)
    return np.ascontiguousarray(g).reshape(-1)


# ----------------------------------------------------------------------------
# Assembly (Sec. 3.1.2) and the constrained system
# ----------------------------------------------------------------------------
def assemble_unconstrained(m: Mesh, gamma: np.ndarray, ngauss: int = 3) -> sp.csr_matrix:
    """J = sum_e [C(gamma_e) Jc + k(gamma_e) Jk], no boundary conditions."""
    ge = element_gamma(m, gamma)
    C = simp_C(m.mat, ge)
    k = simp_k(m.mat, ge)
    Jc, Jk = element_matrices(m.h, m.dt, ngauss)
    conn = element_connectivity(m)
    nv = m.nv
    rows = np.repeat(conn, nv, axis=1).reshape(-1)
    cols = np.tile(conn, (1, nv)).reshape(-1)
    vals = (C[:, None, None] * Jc[None] + k[:, None, None] * Jk[None]).reshape(-1)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m.n_nodes, m.n_nodes))


def constrain(A: sp.spmatrix, dmask: np.ndarray) -> sp.csr_matrix:
    """Rows and columns of prescribed nodes replaced by the identity:
    A_bc = D A D + (I - D), D = diag(free)."""
    free = (~dmask).astype(np.float64)
    D = sp.diags(free)
    return (D @ A @ D + sp.diags(1.0 - free)).tocsr()


def assemble(m: Mesh, gamma: np.ndarray, ngauss: int = 3) -> sp.csr_matrix:
    return constrain(assemble_unconstrained(m, gamma, ngauss), dirichlet_mask(m))


# ----------------------------------------------------------------------------
# Source vector f_i = int N_i Q dV (Sec. 3.1.2), zero at prescribed nodes.
# Reading: the integral uses 2-point Gauss per axis and element; for sources that
# are uniform in space the spatial integral is then exact (the moving Gaussian of
# Example 2 is integrated by the same rule).
# ----------------------------------------------------------------------------
def source_fn(kind: str, q0: float = 1.0, a: float = 1.0, b: float = 0.5, f: float = 4.0,
              center: Tuple[float, float] = (0.5, 0.5)):
    if kind == "uniform":
        return lambda t, *x: q0 * np.ones_like(t)
    if kind == "sin_t":
        return lambda t, *x: q0 * (a + b * np.sin(2.0 * math.pi * f * t))
    if kind == "gaussian":
        # Example 2 (Sec. 2.3.2), two space dimensions: a Gaussian of peak q0 and width
        # sigma = a whose centre moves on a circle of radius R = b about `center` (the middle of
        # the domain) with angular frequency omega = f, starting at angle pi/2 (the top).
        cx, cy = center

        def gauss(t, y, x):
            x1 = cx + b * np.cos(f * t + math.pi / 2.0)
            x2 = cy + b * np.sin(f * t + math.pi / 2.0)
            return q0 * np.exp(-((x - x1) ** 2 + (y - x2) ** 2) / (2.0 * a * a))
        return gauss
    raise ValueError(kind)


def assemble_source(m: Mesh, Q: Callable, nq: int = 2, constrained: bool = True) -> np.ndarray:
    """f_a = sum_e int_e N_a Q dV by nq-point Gauss per axis.  Q(t, [z,] y, x)."""
    sd = m.sd
    gp, gw = gauss_1d(nq)
    conn = element_connectivity(m)
    eidx = np.indices(m.elem_shape).reshape(sd + 1, -1)  # (t, [z], y, x)
    sizes = list(m.h) + [m.dt]
    f = np.zeros(m.n_nodes)
    for q in itertools.product(range(nq), repeat=sd + 1):
        wq = np.prod([gw[qi] * sizes[d] for d, qi in enumerate(q)])
        # physical coordinates of this quadrature point in every element
        t = (eidx[0] + gp[q[sd]]) * m.dt
        xs = [(eidx[sd - d] + gp[q[d]]) * m.h[d] for d in range(sd)]  # x, y, (z)
        Qv = Q(t, *reversed(xs))
        for a in range(m.nv):
            Na = 1.0
            for d in range(sd + 1):
                bit = (a >> d) & 1
                Na *= (1.0 - gp[q[d]]) if bit == 0 else gp[q[d]]
            np.add.at(f, conn[:, a], wq * Na * Qv)
    if constrained:
        f[dirichlet_mask(m)] = 0.0
    return f


def source_rows(m: Mesh, Q: Callable, rows: np.ndarray, nq: int = 2) -> np.ndarray:
    """f_i of assemble_source for the listed nodes only, element by element (for meshes too
    large to assemble): the sum over the elements containing node i of the nq-point Gauss
    integral of N_i Q; prescribed nodes are 0."""
    sd = m.sd
    shape = m.node_shape
    dm = dirichlet_mask(m)
    gp, gw = gauss_1d(nq)
    sizes = list(m.h) + [m.dt]
    out = np.zeros(len(rows))
    for r, node in enumerate(np.asarray(rows)):
        if dm[node]:
            continue
        idx = np.unravel_index(node, shape)  # (t, [z], y, x)
        acc = 0.0
        for e_off in itertools.product((0, 1), repeat=sd + 1):
            e = tuple(i - 1 + o for i, o in zip(idx, e_off))
            if any(v < 0 or v >= n for v, n in zip(e, m.elem_shape)):
                continue
            loc = [i - v for i, v in zip(idx, e)]  # local coordinate bits, (t, [z], y, x)
            for q in itertools.product(range(nq), repeat=sd + 1):  # q[d]: axis d of (x, y, [z], t)
                wq = np.prod([gw[qi] * sizes[d] for d, qi in enumerate(q)])
                t = (e[0] + gp[q[sd]]) * m.dt
                xs = [(e[len(shape) - 1 - d] + gp[q[d]]) * m.h[d] for d in range(sd)]
                Na = 1.0
                for d in range(sd):
                    bit = loc[len(shape) - 1 - d]
                    Na *= (1.0 - gp[q[d]]) if bit == 0 else gp[q[d]]
                Na *= (1.0 - gp[q[sd]]) if loc[0] == 0 else gp[q[sd]]
                acc += wq * Na * float(Q(np.array(t), *reversed([np.array(v) for v in xs])))
        out[r] = acc
    return out


# ----------------------------------------------------------------------------
# Direct solves (the plain definition of what the FGMRES + multigrid solve reaches)
# ----------------------------------------------------------------------------
def factor(A: sp.spmatrix):
    """Sparse LU (SuperLU, minimum-degree ordering on A^T + A)."""
    return spla.splu(sp.csc_matrix(A), permc_spec="MMD_AT_PLUS_A")


def solve_direct(A: sp.spmatrix, b: np.ndarray, lu=None, transpose: bool = False) -> np.ndarray:
    lu = factor(A) if lu is None else lu
    return lu.solve(np.asarray(b), trans="T" if transpose else "N")


def solve_block_tridiag_time(A: sp.spmatrix, b: np.ndarray, nt: int) -> np.ndarray:
    """Direct solve by block elimination in time.  With time the slowest index the
    matrix is block tridiagonal (the M_t coupling reaches one plane forward and one
    back), so Gaussian elimination over the nt+1 plane blocks needs no fill outside them."""
    import scipy.linalg as sl
    A = sp.csr_matrix(A)
    N = A.shape[0]
    P = N // (nt + 1)
    blk = lambda i, j: A[i * P:(i + 1) * P, j * P:(j + 1) * P]
    lus, ys = [sl.lu_factor(blk(0, 0).toarray())], [np.array(b[:P], dtype=A.dtype)]
    for n in range(1, nt + 1):
        Lt = sl.lu_solve(lus[-1], blk(n, n - 1).T.toarray(), trans=1)
        S = blk(n, n).toarray() - (blk(n - 1, n).T @ Lt).T
        ys.append(b[n * P:(n + 1) * P] - Lt.T @ ys[-1])
        lus.append(sl.lu_factor(S))
    x = np.zeros(N, dtype=np.result_type(A.dtype, b.dtype))
    x[nt * P:] = sl.lu_solve(lus[nt], ys[nt])
    for n in range(nt - 1, -1, -1):
        x[n * P:(n + 1) * P] = sl.lu_solve(lus[n], ys[n] - blk(n, n + 1) @ x[(n + 1) * P:(n + 2) * P])
    return x


def solve_dense(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    return np.linalg.solve(A.toarray(), b)


@dataclass
class Solution:
    s: np.ndarray
    f: np.ndarray
    A: sp.csr_matrix
    lu: object = None


def forward(m: Mesh, gamma: np.ndarray, source: str = "uniform", q0: float = 1.0,
            **src) -> Solution:
    A = assemble(m, gamma)
    f = assemble_source(m, source_fn(source, q0, **src))
    lu = factor(A)
    return Solution(solve_direct(A, f, lu), f, A, lu)


# ----------------------------------------------------------------------------
# Objectives and adjoint (Sec. 3.3.1 and 3.3.3)
# ----------------------------------------------------------------------------
def compliance(f: np.ndarray, s: np.ndarray) -> float:
    """Thermal compliance phi = f^T s; d phi / d s = f^T."""
    return float(f @ s)


def pnorm(m: Mesh, s: np.ndarray, P: int = 20):
    """phi = (sum_e T_avg,e^P)^(1/P) with T_avg,e the mean of the element's nodal
    values, and its assembled gradient theta^((1-P)/P) T_avg,e^(P-1) / n_v per
    element node (Sec. 3.3.3; n_v = 8 for (2+1)D elements)."""
    conn = element_connectivity(m)
    Tavg = s[conn].mean(axis=1)
    theta = np.sum(Tavg ** P)
    phi = theta ** (1.0 / P)
    per_e = theta ** ((1.0 - P) / P) * Tavg ** (P - 1) / m.nv
    g = np.zeros_like(s)
    np.add.at(g, conn.reshape(-1), np.repeat(per_e, m.nv))
    return float(phi), g


def adjoint(A: sp.spmatrix, dphids: np.ndarray, dmask: np.ndarray, lu=None) -> np.ndarray:
    """J^T Lambda = (d phi / d s)^T, with Lambda = 0 at prescribed nodes."""
    rhs = np.where(dmask, 0.0, dphids)
    return solve_direct(A, rhs, lu, transpose=True)


def sensitivities(m: Mesh, gamma: np.ndarray, s: np.ndarray, lam: np.ndarray,
                  extruded: Optional[bool] = None) -> np.ndarray:
    """d phi / d gamma_e = - Lambda_e^T (dC/dgamma Jc + dk/dgamma Jk) s_e (Sec. 3.3.3;
    f does not depend on the design).  For an extruded design the element
    sensitivities are summed along time (transpose of the extrusion, Sec. 3.4.1)."""
    ge = element_gamma(m, gamma)
    dC = simp_dC(m.mat, ge)
    dk = simp_dk(m.mat, ge)
    Jc, Jk = element_matrices(m.h, m.dt)
    conn = element_connectivity(m)
    se = s[conn]
    le = lam[conn]
    g = -(dC * np.einsum("ea,ab,eb->e", le, Jc, se) + dk * np.einsum("ea,ab,eb->e", le, Jk, se))
    g = g.reshape(m.elem_shape)
    if extruded is None:
        extruded = np.asarray(gamma).size == int(np.prod(m.ns))
    if extruded:
        return g.sum(axis=0)
    return g


# ----------------------------------------------------------------------------
# Semi-coarsening hierarchy (Algorithm 1) with lambda_crit (Sec. 3.2.1)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Level:
    ns: Tuple[int, ...]
    nt: int
    h: Tuple[float, ...]
    dt: float
    to_next: str = ""  # "space" | "time" | "" (coarsest)

    @property
    def n_nodes(self) -> int:
        n = self.nt + 1
        for k in self.ns:
            n *= k + 1
        return n


def d_eff(mat: Material) -> float:
    """D_eff = sqrt(k_con k_ins / (C_con C_ins))."""
    return math.sqrt(mat.k_con * mat.k_ins / (mat.C_con * mat.C_ins))


def hierarchy(m: Mesh, lam_crit: float = 0.5, n_levels: Optional[int] = None,
              coarse_cap: Optional[int] = None, mode: str = "semi") -> List[Level]:
    """Algorithm 1.  lambda = D_eff dt / dx^2; lambda < lambda_crit -> coarsen time,
    else coarsen space (all spatial axes).  Reading for unequal spatial sizes: dx is
    the smallest spatial element size.  Stop after n_levels levels, or once the
    level has at most coarse_cap nodes.  If the chosen axis cannot be halved
    (odd count, or spatial count below 4 / time count below 2) the other is used;
    if neither can, the hierarchy ends.  mode="full" halves space and time together."""
    D = d_eff(m.mat)
    ns, nt, h, dt = tuple(m.ns), m.nt, tuple(m.h), m.dt
    levels = []
    while True:
        cur = Level(ns, nt, h, dt)
        done = (n_levels is not None and len(levels) + 1 >= n_levels) or \
               (coarse_cap is not None and cur.n_nodes <= coarse_cap)
        can_s = all(n % 2 == 0 and n >= 4 for n in ns)
        can_t = nt % 2 == 0 and nt >= 2
        if mode == "full":
            kind = "full" if (can_s and can_t) else ""
        else:
            lam = D * dt / min(h) ** 2
            kind = "time" if lam < lam_crit else "space"
            if kind == "time" and not can_t:
                kind = "space" if can_s else ""
            elif kind == "space" and not can_s:
                kind = "time" if can_t else ""
        if done or not kind:
            levels.append(cur)
            return levels
        levels.append(Level(ns, nt, h, dt, kind))
        if kind in ("space", "full"):
            ns = tuple(n // 2 for n in ns)
            h = tuple(2 * x for x in h)
        if kind in ("time", "full"):
            nt //= 2
            dt *= 2


# ----------------------------------------------------------------------------
# Transfer operators and Galerkin coarse operators (Sec. 3.2, J_{l+1} = P^T J_l P)
# ----------------------------------------------------------------------------
def interp_1d(nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc+1 coarse nodes to 2nc+1 vertex-nested fine nodes."""
    nf = 2 * nc
    rows, cols, vals = [], [], []
    for i in range(nf + 1):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [i // 2, i // 2 + 1]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf + 1, nc + 1))


def prolongation(fine: Level, coarse: Level) -> sp.csr_matrix:
    """Trilinear space-time interpolation P (fine x coarse), as a Kronecker product
    over the axes (t, [z,] y, x).  Axes that are not coarsened use the identity."""
    facs = []
    if coarse.nt != fine.nt:
        facs.append(interp_1d(coarse.nt))
    else:
        facs.append(sp.identity(fine.nt + 1, format="csr"))
    for nf, nc in zip(reversed(fine.ns), reversed(coarse.ns)):
        facs.append(interp_1d(nc) if nc != nf else sp.identity(nf + 1, format="csr"))
    P = facs[0]
    for F in facs[1:]:
        P = sp.kron(P, F, format="csr")
    return P


def inject_mask(fine_mask: np.ndarray, fine: Level, coarse: Level) -> np.ndarray:
    """Coarse prescribed set: coarse nodes whose coincident fine node is prescribed."""
    shp = (fine.nt + 1,) + tuple(n + 1 for n in reversed(fine.ns))
    M = fine_mask.reshape(shp)
    sl = [slice(None, None, 2) if coarse.nt != fine.nt else slice(None)]
    for nf, nc in zip(reversed(fine.ns), reversed(coarse.ns)):
        sl.append(slice(None, None, 2) if nc != nf else slice(None))
    return np.ascontiguousarray(M[tuple(sl)]).reshape(-1)


def galerkin(A: sp.spmatrix, P: sp.spmatrix, fmask: np.ndarray, cmask: np.ndarray):
    """Reading (Dirichlet in Galerkin): A_c = Pt^T A Pt + (I - D_c), with the
    masked prolongation Pt = D_f P D_c, so prescribed nodes stay prescribed on
    every level.  Returns (A_c, Pt)."""
    Df = sp.diags((~fmask).astype(np.float64))
    Dc = sp.diags((~cmask).astype(np.float64))
    Pt = (Df @ P @ Dc).tocsr()
    Ac = (Pt.T @ A @ Pt + sp.diags(cmask.astype(np.float64))).tocsr()
    return Ac, Pt


@dataclass
class MGLevel:
    level: Level
    A: sp.csr_matrix
    mask: np.ndarray
    Pt: Optional[sp.csr_matrix] = None  # masked prolongation from the next coarser level


def build_mg(m: Mesh, gamma: np.ndarray, levels: List[Level]) -> List[MGLevel]:
    A0 = assemble(m, gamma)
    mask0 = dirichlet_mask(m)
    out = [MGLevel(levels[0], A0, mask0)]
    for l in range(1, len(levels)):
        fine, coarse = levels[l - 1], levels[l]
        P = prolongation(fine, coarse)
        cmask = inject_mask(out[-1].mask, fine, coarse)
        Ac, Pt = galerkin(out[-1].A, P, out[-1].mask, cmask)
        out[-1].Pt = Pt
        out.append(MGLevel(coarse, Ac, cmask))
    return out


# ----------------------------------------------------------------------------
# Jacobi-preconditioned GMRES smoother and the V-cycle (Sec. 3.2).
# Reading: right Jacobi preconditioning, exactly m iterations, no early exit
# except an exact breakdown; pre-smoothing starts from zero, post-smoothing
# from the current iterate; the coarsest level is solved directly.
# ----------------------------------------------------------------------------
def gmres_jacobi(A: sp.spmatrix, b: np.ndarray, x0: np.ndarray, m: int = 10,
                 breakdown_tol: float = 0.0, dtype=np.float64) -> np.ndarray:
    """m steps of GMRES on A D^{-1} y = b - A x0, x = x0 + D^{-1} y (Arnoldi with
    modified Gram-Schmidt, least squares by numpy.linalg.lstsq).

    dtype selects the arithmetic: float64 (the oracle proper) or float32, which runs the
    same algorithm with every vector operation in IEEE single precision (matrix entries,
    D^{-1}, matrix-vector products, dot products, norms and updates all float32; the
    (m+1) x m least-squares problem is solved by numpy in float64 and rounded back), to
    measure how far a single-precision smoother lands from the float64 one."""
    A = sp.csr_matrix(A).astype(dtype)
    b = np.asarray(b).astype(dtype)
    x0 = np.asarray(x0).astype(dtype)
    dinv = (dtype(1.0) / A.diagonal()).astype(dtype)
    r = b - A @ x0
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return x0.copy()
    n = b.size
    V = np.zeros((m + 1, n), dtype=dtype)
    H = np.zeros((m + 1, m), dtype=dtype)
    V[0] = r / beta
    k = m
    for j in range(m):
        w = A @ (dinv * V[j])
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= breakdown_tol * beta:
            k = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    e1 = np.zeros(k + 1, dtype=dtype)
    e1[0] = beta
    y = np.linalg.lstsq(H[: k + 1, :k], e1, rcond=None)[0].astype(dtype)
    return x0 + dinv * (V[:k].T @ y)


# A cheaper smoother, one of the variants the paper's outlook names (Sec. 6, "cheaper
# smoothers"): damped (weighted) Jacobi, x <- x + omega D^{-1} (b - A x), nu sweeps.
# Reading: the same nu for pre- and post-smoothing, pre-smoothing from zero (its first sweep
# is x = omega D^{-1} b), omega fixed per hierarchy, 0.5 by default: with 0.7 the V-cycle of a
# space-time design diverges (pinned in the tests).
def jacobi_smooth(A: sp.spmatrix, b: np.ndarray, x0: np.ndarray, nu: int, omega: float,
                  dtype=np.float64) -> np.ndarray:
    """nu damped Jacobi sweeps from x0 (every vector operation in dtype)."""
    A = sp.csr_matrix(A).astype(dtype)
    dinv = (dtype(1.0) / A.diagonal()).astype(dtype)
    x = np.asarray(x0).astype(dtype)
    b = np.asarray(b).astype(dtype)
    w = dtype(omega)
    for _ in range(nu):
        x = x + w * (dinv * (b - A @ x))
    return x


def vcycle(mg: List[MGLevel], b: np.ndarray, l: int = 0, nsmooth: int = 10,
           transpose: bool = False, dtype=np.float64, smoother: str = "gmres",
           omega: float = 0.5) -> np.ndarray:
    """One V-cycle for A_l x = b (A_l^T for transpose=True, which uses the same
    hierarchy since (P^T A P)^T = P^T A^T P).

    dtype = float32 runs the smoothing, residuals and transfers in single precision and
    keeps the coarsest solve in float64 (its result rounded to float32), the precision
    split of a mixed-precision multigrid; float64 is the oracle proper.  smoother "gmres"
    is the paper's Jacobi-GMRES(nsmooth); "jacobi" takes nsmooth damped Jacobi sweeps."""
    A = mg[l].A.T.tocsr() if transpose else mg[l].A
    b = np.asarray(b).astype(dtype)
    if l == len(mg) - 1:
        return np.linalg.solve(A.toarray(), b.astype(np.float64)).astype(dtype)
    A = sp.csr_matrix(A).astype(dtype)

    def smooth(x0):
        if smoother == "jacobi":
            return jacobi_smooth(A, b, x0, nsmooth, omega, dtype=dtype)
        return gmres_jacobi(A, b, x0, nsmooth, dtype=dtype)
    x = smooth(np.zeros_like(b))
    r = b - A @ x
    Pt = mg[l].Pt.astype(dtype)
    xc = vcycle(mg, Pt.T @ r, l + 1, nsmooth, transpose, dtype, smoother, omega)
    x = x + Pt @ xc
    return smooth(x)


def abs_operator(m: Mesh, gamma: np.ndarray, ngauss: int = 3) -> sp.csr_matrix:
    """Element-wise absolute operator |J|_elem = sum_e |C_e Jc| + |k_e Jk| (entry-wise
    absolute values of each element's capacity and conductivity parts, summed without
    cancellation), with the identity on prescribed rows and columns as in assemble().
    It bounds the rounding error of any evaluation of J x that forms the element terms
    and adds them: |fl(J x) - J x| <= c u |J|_elem |x| (componentwise, c a small multiple
    of the number of terms, u the unit roundoff)."""
    ge = element_gamma(m, gamma)
    C = np.abs(simp_C(m.mat, ge))
    k = np.abs(simp_k(m.mat, ge))
    Jc, Jk = element_matrices(m.h, m.dt, ngauss)
    conn = element_connectivity(m)
    nv = m.nv
    rows = np.repeat(conn, nv, axis=1).reshape(-1)
    cols = np.tile(conn, (1, nv)).reshape(-1)
    vals = (C[:, None, None] * np.abs(Jc)[None] + k[:, None, None] * np.abs(Jk)[None]).reshape(-1)
    B = sp.csr_matrix((vals, (rows, cols)), shape=(m.n_nodes, m.n_nodes))
    return constrain(B, dirichlet_mask(m))


# ----------------------------------------------------------------------------
# Single rows of the constrained system, for checks on meshes too large to assemble.
# ----------------------------------------------------------------------------
def apply_rows(m: Mesh, gamma: np.ndarray, x: np.ndarray, rows: np.ndarray,
               absolute: bool = False) -> np.ndarray:
    """(A x)_i for the listed nodes i, element by element: the sum over the elements that
    contain node i of row a(i) of C_e Jc + k_e Jk applied to the element's (masked) values;
    prescribed rows are the identity.  absolute=True gives the same rows of abs_operator
    applied to |x| instead (|C_e Jc| + |k_e Jk| per element, no cancellation)."""
    if absolute:
        x = np.abs(x)
    sd = m.sd
    shape = m.node_shape
    dm = dirichlet_mask(m)
    Jc, Jk = element_matrices(m.h, m.dt)
    ge_shape = m.elem_shape
    g = np.asarray(gamma)
    extruded = g.size == int(np.prod(m.ns))
    g = g.reshape(tuple(reversed(m.ns)) if extruded else ge_shape)
    out = np.zeros(len(rows))
    for r, node in enumerate(np.asarray(rows)):
        if dm[node]:
            out[r] = x[node]
            continue
        idx = np.unravel_index(node, shape)  # (t, [z], y, x)
        acc = 0.0
        for e_off in itertools.product((0, 1), repeat=sd + 1):  # element = node - 1 + offset
            e = tuple(i - 1 + o for i, o in zip(idx, e_off))
            if any(v < 0 or v >= n for v, n in zip(e, ge_shape)):
                continue
            gm = g[e[1:]] if extruded else g[e]
            C, k = simp_C(m.mat, gm), simp_k(m.mat, gm)
            # local index of the node inside element e: bit d of spatial d, top bit time
            loc = [i - v for i, v in zip(idx, e)]
            a = loc[0] << sd
            for d in range(sd):
                a |= loc[len(shape) - 1 - d] << d
            for b in range(m.nv):
                bi = [0] * len(shape)
                bi[0] = e[0] + ((b >> sd) & 1)
                for d in range(sd):
                    bi[len(shape) - 1 - d] = e[len(shape) - 1 - d] + ((b >> d) & 1)
                q = np.ravel_multi_index(tuple(bi), shape)
                if dm[q]:
                    continue
                if absolute:
                    acc += (abs(C * Jc[a, b]) + abs(k * Jk[a, b])) * x[q]
                else:
                    acc += (C * Jc[a, b] + k * Jk[a, b]) * x[q]
        out[r] = acc
    return out


# ----------------------------------------------------------------------------
# PDE filter and Heaviside projection (Sec. 3.3.2).
# The filter solves  -div(D grad psi) + psi = gamma  over the space-time domain, D = diag(
# r_x^2/12 per spatial axis, r_t^2/12 in time), natural boundary conditions on every face.
# Reading: it is discretised with the same trilinear space-time elements as the state: nodal
# psi, (M_f + K_f) psi = T gamma with T_ie = int_e N_i (the element's volume / n_v), and the
# filtered element value is the mean of the element's nodal values, gamma~ = E psi.  An extruded
# (time-constant) design gives a time-constant psi, equal to the spatial filter of one slab.
# ----------------------------------------------------------------------------
def filter_element_matrix(h: Sequence[float], dt: float, r_x: float, r_t: float, ngauss: int = 3) -> np.ndarray:
    """int N_a N_b + sum_d D_dd dN_a/dxi_d dN_b/dxi_d on one h x ... x dt brick (Gauss quadrature)."""
    sd = len(h)
    nv = 2 ** (sd + 1)
    gp, gw = gauss_1d(ngauss)
    sizes = list(h) + [dt]
    D = [r_x ** 2 / 12.0] * sd + [r_t ** 2 / 12.0]
    Ke = np.zeros((nv, nv))
    for q in itertools.product(range(ngauss), repeat=sd + 1):
        wq = np.prod([gw[qi] * sizes[d] for d, qi in enumerate(q)])
        N = np.ones(nv)
        dN = np.ones((sd + 1, nv))
        for a in range(nv):
            for d in range(sd + 1):
                bit = (a >> d) & 1
                phi, dphi = _basis_1d(gp[q[d]])
                N[a] *= phi[bit]
                for dd in range(sd + 1):
                    dN[dd, a] *= (dphi[bit] / sizes[d]) if dd == d else phi[bit]
        Ke += wq * np.outer(N, N)
        for d in range(sd + 1):
            Ke += wq * D[d] * np.outer(dN[d], dN[d])
    return Ke


def filter_operator(m: Mesh, r_x: float, r_t: float) -> sp.csr_matrix:
    """Assembled filter matrix M_f + K_f on the nodes of m (no prescribed nodes)."""
    Ke = filter_element_matrix(m.h, m.dt, r_x, r_t)
    conn = element_connectivity(m)
    nv = m.nv
    rows = np.repeat(conn, nv, axis=1).reshape(-1)
    cols = np.tile(conn, (1, nv)).reshape(-1)
    vals = np.broadcast_to(Ke, (m.n_elem, nv, nv)).reshape(-1)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m.n_nodes, m.n_nodes))


def element_to_node(m: Mesh) -> sp.csr_matrix:
    """T (nodes x elements): T_ie = int_e N_i = v_e / n_v for the nodes i of element e."""
    conn = element_connectivity(m)
    ve = float(np.prod(m.h)) * m.dt
    rows = conn.reshape(-1)
    cols = np.repeat(np.arange(m.n_elem), m.nv)
    return sp.csr_matrix((np.full(rows.size, ve / m.nv), (rows, cols)), shape=(m.n_nodes, m.n_elem))


def node_to_element(m: Mesh) -> sp.csr_matrix:
    """E (elements x nodes): the mean of the element's n_v nodal values."""
    conn = element_connectivity(m)
    rows = np.repeat(np.arange(m.n_elem), m.nv)
    return sp.csr_matrix((np.full(rows.size, 1.0 / m.nv), (rows, conn.reshape(-1))), shape=(m.n_elem, m.n_nodes))


def _filter_mesh(m: Mesh, gamma: np.ndarray) -> Tuple[Mesh, bool]:
    extruded = np.asarray(gamma).size == int(np.prod(m.ns))
    return (with_size(m, m.ns, 1) if extruded else m), extruded


def pde_filter(m: Mesh, gamma: np.ndarray, r_x: float, r_t: float) -> np.ndarray:
    """gamma~ = E (M_f + K_f)^-1 T gamma (direct sparse solve), same layout as gamma."""
    fm, extruded = _filter_mesh(m, gamma)
    g = np.asarray(gamma, dtype=np.float64).reshape(-1)
    A = filter_operator(fm, r_x, r_t)
    psi = solve_direct(A, element_to_node(fm) @ g)
    return (node_to_element(fm) @ psi).reshape(np.asarray(gamma).shape)


def heaviside(x: np.ndarray, beta: float = 32.0, eta: float = 0.5) -> np.ndarray:
    """Projection of Sec. 3.3.2: (tanh(beta eta) + tanh(beta (x - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)))."""
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return (np.tanh(beta * eta) + np.tanh(beta * (np.asarray(x) - eta))) / den


def heaviside_derivative(x: np.ndarray, beta: float = 32.0, eta: float = 0.5) -> np.ndarray:
    """d heaviside / dx = beta (1 - tanh^2(beta (x - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)))."""
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return beta * (1.0 - np.tanh(beta * (np.asarray(x) - eta)) ** 2) / den


def design_chain(m: Mesh, gamma: np.ndarray, r_x: float, r_t: float, beta: float = 32.0, eta: float = 0.5):
    """Physical design gamma_bar = H(F gamma) and gamma~ = F gamma."""
    gt = pde_filter(m, gamma, r_x, r_t)
    return heaviside(gt, beta, eta), gt


def chain_rule(m: Mesh, dphi_dphys: np.ndarray, gamma_tilde: np.ndarray, r_x: float, r_t: float,
               beta: float = 32.0, eta: float = 0.5) -> np.ndarray:
    """d phi / d gamma = F^T (H'(gamma~) * d phi / d gamma_bar).  F = E A^-1 T with T = v_e E^T and
    A symmetric, so F^T = F: the sensitivities pass through the same filter (Sec. 3.3.2)."""
    return pde_filter(m, heaviside_derivative(gamma_tilde, beta, eta) * dphi_dphys, r_x, r_t)


# ----------------------------------------------------------------------------
# Method of Moving Asymptotes (Svanberg 1987) for one constraint g1(x) <= 0, the
# optimiser named in Sec. 3.3.3 (volume constraint of Sec. 3.3.1).  Readings (the
# paper cites a modified form of Guest et al.'s initial asymptotes without values):
# - asymptotes: the first two iterations at x -/+ MMA_S0 (x_max - x_min); later
#   ones move by MMA_INCR where the last two steps kept their sign and MMA_DECR
#   where it flipped, kept within 0.01 .. 10 (x_max - x_min) of x;
# - bounds of the subproblem: alpha = max(x_min, L + 0.1 (x - L), x - MMA_MOVE span),
#   beta = min(x_max, U - 0.1 (U - x), x + MMA_MOVE span);
# - the convex approximations of Svanberg's later formulation:
#   p = (U - x)^2 (1.001 df+ + 0.001 df- + MMA_RAA / span),
#   q = (x - L)^2 (0.001 df+ + 1.001 df- + MMA_RAA / span);
# - the subproblem solved through its dual: for a multiplier lam >= 0 each x_j
#   minimises P_j / (U_j - x) + Q_j / (x - L_j) with P = p0 + lam p1, Q = q0 + lam q1,
#   x_j = (sqrt(P) L + sqrt(Q) U) / (sqrt(P) + sqrt(Q)) clipped to [alpha, beta];
#   lam = 0 when the approximated constraint holds there, else the root of the
#   approximated constraint (decreasing in lam), by bisection; when it cannot be met
#   inside [alpha, beta] (the paper's volume constraint only from an infeasible start),
#   lam stops at MMA_LAM_MAX, the most feasible point of the subproblem.
# ----------------------------------------------------------------------------
MMA_S0, MMA_INCR, MMA_DECR, MMA_MOVE, MMA_RAA, MMA_LAM_MAX = 0.05, 1.2, 0.7, 0.2, 1e-5, 1e40


def mma_asymptotes(it: int, x, xold1, xold2, low, upp, xmin: float = 0.0, xmax: float = 1.0):
    """Asymptotes L, U of iteration it (1-based) of the readings above."""
    span = xmax - xmin
    if it <= 2:
        return x - MMA_S0 * span, x + MMA_S0 * span
    sgn = (x - xold1) * (xold1 - xold2)
    fac = np.where(sgn > 0, MMA_INCR, np.where(sgn < 0, MMA_DECR, 1.0))
    low = np.clip(x - fac * (xold1 - low), x - 10.0 * span, x - 0.01 * span)
    upp = np.clip(x + fac * (upp - xold1), x + 0.01 * span, x + 10.0 * span)
    return low, upp


def mma_subproblem(x, low, upp, df0, g1: float, dg1, xmin: float = 0.0, xmax: float = 1.0):
    """The convex separable subproblem at x: bounds alpha, beta and the terms p0, q0, p1, q1, r1
    of f0 ~ sum p0 / (U - x) + q0 / (x - L) and g1 ~ sum p1 / (U - x) + q1 / (x - L) + r1."""
    span = xmax - xmin
    alpha = np.maximum(np.maximum(xmin, low + 0.1 * (x - low)), x - MMA_MOVE * span)
    beta = np.minimum(np.minimum(xmax, upp - 0.1 * (upp - x)), x + MMA_MOVE * span)
    ux2, xl2 = (upp - x) ** 2, (x - low) ** 2
    reg = MMA_RAA / span

    def pq(d):
        dp, dm = np.maximum(d, 0.0), np.maximum(-d, 0.0)
        return ux2 * (1.001 * dp + 0.001 * dm + reg), xl2 * (0.001 * dp + 1.001 * dm + reg)
    p0, q0 = pq(np.asarray(df0, dtype=np.float64))
    p1, q1 = pq(np.asarray(dg1, dtype=np.float64))
    r1 = g1 - np.sum(p1 / (upp - x) + q1 / (x - low))
    return alpha, beta, p0, q0, p1, q1, r1


def mma_x_of(lam: float, low, upp, alpha, beta, p0, q0, p1, q1):
    """The subproblem's minimiser for multiplier lam (closed form, clipped)."""
    sp_, sq_ = np.sqrt(p0 + lam * p1), np.sqrt(q0 + lam * q1)
    return np.clip((sp_ * low + sq_ * upp) / (sp_ + sq_), alpha, beta)


def mma_update(it: int, x, xold1, xold2, low, upp, df0, g1: float, dg1, xmin: float = 0.0,
               xmax: float = 1.0, rel_tol: float = 1e-15):
    """One MMA iteration: returns (x_new, L, U, lam)."""
    x = np.asarray(x, dtype=np.float64)
    low, upp = mma_asymptotes(it, x, xold1, xold2, low, upp, xmin, xmax)
    alpha, beta, p0, q0, p1, q1, r1 = mma_subproblem(x, low, upp, df0, g1, dg1, xmin, xmax)

    def g_of(lam):
        xs = mma_x_of(lam, low, upp, alpha, beta, p0, q0, p1, q1)
        return np.sum(p1 / (upp - xs) + q1 / (xs - low)) + r1
    lam = 0.0
    if g_of(0.0) > 0.0:
        lo, hi = 0.0, 1.0
        while g_of(hi) > 0.0 and hi < MMA_LAM_MAX:
            lo, hi = hi, 2.0 * hi
        while hi - lo > rel_tol * hi:
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            if g_of(mid) > 0.0:
                lo = mid
            else:
                hi = mid
        lam = hi
    return mma_x_of(lam, low, upp, alpha, beta, p0, q0, p1, q1), low, upp, lam


# ----------------------------------------------------------------------------
# One design iteration of the optimisation problem (Sec. 3.3): the nested formulation solves the
# state for the current design, then the objective (Sec. 3.3.1) and its adjoint, the
# sensitivities with respect to the physical design (Sec. 3.3.3), the chain rule through the
# projection and the filter (Sec. 3.3.2), the volume constraint and its gradient, and one MMA
# step on gamma in [0, 1].  Readings:
# - the volume constraint is taken on the physical design gamma_bar, so its gradient passes
#   through the projection and the filter like the objective's;
# - uniform elements: chi = mean(gamma_bar) / v_f - 1 and d chi / d gamma_bar_e = 1 / (v_f N_e);
# - the objective enters MMA as TO_OBJ_SCALE * phi / phi_1, phi_1 its value at the first
#   iteration (the paper gives no scaling; MMA's fixed regularisation needs one).
# ----------------------------------------------------------------------------
TO_OBJ_SCALE = 10.0


def volume_constraint(gamma_bar: np.ndarray, vf: float):
    """chi = sum_e gamma_bar_e v_e / (v_f |Pi|) - 1 and d chi / d gamma_bar (Sec. 3.3.1, 3.3.3)."""
    g = np.asarray(gamma_bar, dtype=np.float64)
    return float(g.mean() / vf - 1.0), np.full(g.shape, 1.0 / (vf * g.size))


def topopt_gradients(m: Mesh, gamma: np.ndarray, vf: float, r_x: float, r_t: float, beta: float = 32.0,
                     eta: float = 0.5, objective: str = "pnorm", P: int = 20, source: str = "uniform",
                     q0: float = 1.0, **src) -> dict:
    """phi, chi and their gradients with respect to the design variables gamma (filter and
    projection included), with the intermediate fields."""
    gb, gt = design_chain(m, gamma, r_x, r_t, beta, eta)
    sol = forward(m, gb, source, q0, **src)
    if objective == "pnorm":
        phi, dphids = pnorm(m, sol.s, P)
    else:
        phi, dphids = compliance(sol.f, sol.s), sol.f
    lam = adjoint(sol.A, dphids, dirichlet_mask(m), sol.lu)
    dphys = sensitivities(m, gb, sol.s, lam)
    chi, dchi_phys = volume_constraint(gb, vf)
    return dict(phi=phi, chi=chi, dphi=chain_rule(m, dphys, gt, r_x, r_t, beta, eta),
                dchi=chain_rule(m, dchi_phys, gt, r_x, r_t, beta, eta), gamma_tilde=gt, gamma_bar=gb,
                s=sol.s, lam=lam)


@dataclass
class TopOptHistory:
    """What the loop carries from one iteration to the next: the iteration count, phi_1 and the
    MMA history (two previous iterates, asymptotes)."""
    it: int = 0
    phi1: float = 0.0
    xold1: Optional[np.ndarray] = None
    xold2: Optional[np.ndarray] = None
    low: Optional[np.ndarray] = None
    upp: Optional[np.ndarray] = None


def topopt_step(m: Mesh, gamma: np.ndarray, hist: TopOptHistory, vf: float, r_x: float, r_t: float,
                **kw) -> Tuple[np.ndarray, dict]:
    """One design iteration from gamma: returns the next design and the iteration's fields
    (phi and chi at gamma, gradients, the MMA multiplier lam_mma)."""
    d = topopt_gradients(m, gamma, vf, r_x, r_t, **kw)
    x = np.asarray(gamma, dtype=np.float64).reshape(-1)
    if hist.it == 0:
        hist.phi1 = d["phi"]
        hist.xold1 = hist.xold2 = hist.low = hist.upp = np.zeros_like(x)
    hist.it += 1
    df0 = (TO_OBJ_SCALE / hist.phi1) * d["dphi"].reshape(-1)
    xn, low, upp, lam = mma_update(hist.it, x, hist.xold1, hist.xold2, hist.low, hist.upp, df0, d["chi"],
                                   d["dchi"].reshape(-1))
    hist.xold2, hist.xold1, hist.low, hist.upp = hist.xold1, x.copy(), low, upp
    d["lam_mma"] = lam
    d["df0"] = df0
    return xn.reshape(np.shape(gamma)), d


# ----------------------------------------------------------------------------
# Reference time stepping (Sec. 4): the comparison solver takes first-order backward
# differences (BDF1) in time on the spatial mesh.  Reading: consistent, capacity-weighted mass,
#   (M_C + dt K_k) T^{n+1} = M_C T^n + dt F(t_{n+1}),   T^0 = 0,
# with M_C = sum_e C_e M_e and K_k = sum_e k_e K_e from the design of slab n (a space-time design
# changes from step to step), F_i(t) = int N_i Q(t, x) dx by 2-point Gauss per axis, and the
# spatial sink prescribed (T = 0) at every step.
# ----------------------------------------------------------------------------
def spatial_element_matrices(h: Sequence[float], ngauss: int = 2) -> Tuple[np.ndarray, np.ndarray]:
    """int N_a N_b and int grad N_a . grad N_b on one h_1 x ... brick (Gauss quadrature, exact
    for these multilinear products with 2 points)."""
    sd = len(h)
    nv = 2 ** sd
    gp, gw = gauss_1d(ngauss)
    Me = np.zeros((nv, nv))
    Ke = np.zeros((nv, nv))
    for q in itertools.product(range(ngauss), repeat=sd):
        wq = np.prod([gw[qi] * h[d] for d, qi in enumerate(q)])
        N = np.ones(nv)
        dN = np.ones((sd, nv))
        for a in range(nv):
            for d in range(sd):
                phi, dphi = _basis_1d(gp[q[d]])
                bit = (a >> d) & 1
                N[a] *= phi[bit]
                for dd in range(sd):
                    dN[dd, a] *= (dphi[bit] / h[d]) if dd == d else phi[bit]
        Me += wq * np.outer(N, N)
        Ke += wq * dN.T @ dN
    return Me, Ke


def spatial_connectivity(m: Mesh) -> np.ndarray:
    """conn[e, a] = spatial node of local node a (bits x, y, [z]) of spatial element e; the
    spatial node numbering is that of one time plane."""
    return element_connectivity(with_size(m, m.ns, 1))[:, : 2 ** m.sd]


def bdf1_matrices(m: Mesh, gamma_slab: np.ndarray) -> Tuple[sp.csr_matrix, sp.csr_matrix]:
    """M_C and K_k on the spatial nodes for one slab's design (spatial element order)."""
    Me, Ke = spatial_element_matrices(m.h)
    conn = spatial_connectivity(m)
    ge = np.asarray(gamma_slab, dtype=np.float64).reshape(-1)
    nv = conn.shape[1]
    n_sp = int(np.prod([n + 1 for n in m.ns]))
    rows = np.repeat(conn, nv, axis=1).reshape(-1)
    cols = np.tile(conn, (1, nv)).reshape(-1)
    C = simp_C(m.mat, ge)
    k = simp_k(m.mat, ge)
    Mc = sp.csr_matrix(((C[:, None, None] * Me[None]).reshape(-1), (rows, cols)), shape=(n_sp, n_sp))
    Kk = sp.csr_matrix(((k[:, None, None] * Ke[None]).reshape(-1), (rows, cols)), shape=(n_sp, n_sp))
    return Mc, Kk


def bdf1_load(m: Mesh, Q: Callable, t: float, nq: int = 2) -> np.ndarray:
    """F_i(t) = int N_i(x) Q(t, x) dx by nq-point Gauss per axis."""
    sd = m.sd
    gp, gw = gauss_1d(nq)
    conn = spatial_connectivity(m)
    eidx = np.indices(tuple(reversed(m.ns))).reshape(sd, -1)  # ([z], y, x)
    F = np.zeros(int(np.prod([n + 1 for n in m.ns])))
    for q in itertools.product(range(nq), repeat=sd):
        wq = np.prod([gw[qi] * m.h[d] for d, qi in enumerate(q)])
        xs = [(eidx[sd - 1 - d] + gp[q[d]]) * m.h[d] for d in range(sd)]  # x, y, (z)
        Qv = Q(np.full(eidx.shape[1], t), *reversed(xs))
        for a in range(2 ** sd):
            Na = 1.0
            for d in range(sd):
                Na *= (1.0 - gp[q[d]]) if ((a >> d) & 1) == 0 else gp[q[d]]
            np.add.at(F, conn[:, a], wq * Na * Qv)
    return F


def bdf1_forward(m: Mesh, gamma: np.ndarray, source: str = "uniform", q0: float = 1.0, **src) -> np.ndarray:
    """BDF1 trajectory T (nt + 1 planes of spatial nodes, plane n at t = n dt), direct sparse
    solve per step."""
    Q = source_fn(source, q0, **src)
    n_sp = int(np.prod([n + 1 for n in m.ns]))
    dm = dirichlet_mask(m).reshape(m.nt + 1, n_sp)[1]
    eg = element_gamma(m, gamma).reshape(m.nt, -1)
    extruded = np.asarray(gamma).size == int(np.prod(m.ns))
    keep = sp.diags((~dm).astype(np.float64))
    T = np.zeros(n_sp)
    traj = [T]
    lu = Mc = None
    for n in range(m.nt):
        if lu is None or not extruded:
            Mc, Kk = bdf1_matrices(m, eg[n])
            A = (keep @ (Mc + m.dt * Kk) @ keep + sp.diags(dm.astype(np.float64))).tocsr()
            lu = factor(A)
        r = Mc @ T + m.dt * bdf1_load(m, Q, (n + 1) * m.dt)
        r[dm] = 0.0
        T = solve_direct(A, r, lu)
        traj.append(T)
    return np.array(traj)


def bdf1_adjoint(m: Mesh, gamma: np.ndarray, traj: np.ndarray, P: int = 20):
    """Discrete adjoint of bdf1_forward for the p-norm objective of Sec. 3.3.1 taken over the
    space-time elements of the trajectory.  Step n is the constraint
    A_n T^{n+1} - M_n T^n - dt F^{n+1} = 0 (A_n = M_C + dt K_k of slab n, prescribed rows and
    columns removed), so the multipliers solve, from the last step backwards,
      A_{m-1} Lambda^m = d phi / d T^m + M_m Lambda^{m+1},   Lambda^{N+1} = 0,
    zero at prescribed nodes, and for element e of slab n
      d phi / d gamma_e = -Lambda^{n+1}_e . (C'_e M_e (T^{n+1} - T^n)_e + dt k'_e K_e T^{n+1}_e),
    summed over the slabs for an extruded design.  Returns (phi, Lambda, sensitivities)."""
    n_sp = int(np.prod([n + 1 for n in m.ns]))
    traj = np.asarray(traj, dtype=np.float64).reshape(m.nt + 1, n_sp)
    phi, dphids = pnorm(m, traj.reshape(-1), P)
    g = dphids.reshape(m.nt + 1, n_sp)
    dm = dirichlet_mask(m).reshape(m.nt + 1, n_sp)[1]
    keep = sp.diags((~dm).astype(np.float64))
    eg = element_gamma(m, gamma).reshape(m.nt, -1)
    lam = np.zeros((m.nt + 2, n_sp))
    for mm_ in range(m.nt, 0, -1):
        Mc_prev, Kk_prev = bdf1_matrices(m, eg[mm_ - 1])
        A = (keep @ (Mc_prev + m.dt * Kk_prev) @ keep + sp.diags(dm.astype(np.float64))).tocsr()
        r = g[mm_].copy()
        if mm_ < m.nt:
            Mc_next, _ = bdf1_matrices(m, eg[mm_])
            r += Mc_next @ lam[mm_ + 1]
        r[dm] = 0.0
        lam[mm_] = solve_direct(A, r)
    Me, Ke = spatial_element_matrices(m.h)
    conn = spatial_connectivity(m)
    dC = simp_dC(m.mat, eg)
    dk = simp_dk(m.mat, eg)
    sens = np.zeros((m.nt, conn.shape[0]))
    for n in range(m.nt):
        le = lam[n + 1][conn]
        dT = (traj[n + 1] - traj[n])[conn]
        T1 = traj[n + 1][conn]
        sens[n] = -(dC[n] * np.einsum("ea,ab,eb->e", le, Me, dT) +
                    m.dt * dk[n] * np.einsum("ea,ab,eb->e", le, Ke, T1))
    sens = sens.reshape(m.elem_shape)
    if np.asarray(gamma).size == int(np.prod(m.ns)):
        sens = sens.sum(axis=0)
    return phi, lam[: m.nt + 1], sens
