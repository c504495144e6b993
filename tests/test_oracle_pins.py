"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms
derived by hand, textbook 1D finite-element matrices combined by Kronecker
products, brute-force integration of global hat functions, exact discrete
solutions, conservation, convergence orders, the hierarchies printed in the
paper, finite differences and complex-step derivatives.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import st_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UNITCAP = O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


# ---------------------------------------------------------------- textbook 1D matrices
def mass1(h):
    return h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])


def stiff1(h):
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


UPWIND = np.array([[0.0, 0.0], [-1.0, 1.0]])


def kron_all(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.kron(out, m)
    return out


def glob_mass(n, h):
    d = np.full(n + 1, 4.0); d[0] = d[-1] = 2.0
    return sp.diags([np.full(n, 1.0), d, np.full(n, 1.0)], [-1, 0, 1]) * (h / 6.0)


def glob_stiff(n, h):
    d = np.full(n + 1, 2.0); d[0] = d[-1] = 1.0
    return sp.diags([np.full(n, -1.0), d, np.full(n, -1.0)], [-1, 0, 1]) / h


def glob_upwind(n):
    d = np.ones(n + 1); d[0] = 0.0
    return sp.diags([-np.ones(n), d], [-1, 0])


def kron_spatial_mass_stiff(ns, hs):
    """Global spatial mass and stiffness for Q1 on a tensor grid, axes (z, y, x)."""
    Ms = [glob_mass(n, h) for n, h in zip(reversed(ns), reversed(hs))]
    Ks = [glob_stiff(n, h) for n, h in zip(reversed(ns), reversed(hs))]
    M = Ms[0]
    for X in Ms[1:]:
        M = sp.kron(M, X)
    K = None
    for d in range(len(ns)):
        term = Ks[0] if d == 0 else Ms[0]
        for e in range(1, len(ns)):
            term = sp.kron(term, Ks[e] if e == d else Ms[e])
        K = term if K is None else K + term
    return M.tocsr(), K.tocsr()


# ---------------------------------------------------------------- SIMP
def test_simp_endpoints_and_derivatives():
    m = O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
    assert O.simp_C(m, 0.0) == 0.5 and O.simp_C(m, 1.0) == 1.0
    assert O.simp_k(m, 0.0) == 0.03 and O.simp_k(m, 1.0) == 3.0
    g = np.linspace(0.05, 0.95, 7)
    h = 1e-6
    np.testing.assert_allclose(O.simp_dC(m, g), (O.simp_C(m, g + h) - O.simp_C(m, g - h)) / (2 * h), rtol=1e-8)
    np.testing.assert_allclose(O.simp_dk(m, g), (O.simp_k(m, g + h) - O.simp_k(m, g - h)) / (2 * h), rtol=1e-8)
    np.testing.assert_allclose(O.simp_k(m, 0.5), 0.03 + 2.97 * 0.125)


# ---------------------------------------------------------------- P1 element closed form
@pytest.mark.parametrize("h,dt", [((0.25, 0.25), 0.1), ((0.1, 0.3), 0.07), ((0.2, 0.5, 0.125), 0.3)])
def test_element_matrices_kronecker_closed_form(h, dt):
    """With k_ad = C dt / 2 the capacity part is exactly upwind (x) spatial mass and the
    conductivity part is time mass (x) spatial stiffness."""
    Jc, Jk = O.element_matrices(h, dt)
    sd = len(h)
    Ms = [mass1(x) for x in reversed(h)]
    Ks = [stiff1(x) for x in reversed(h)]
    Mx = kron_all(*Ms)
    Kx = sum(kron_all(*[Ks[e] if e == d else Ms[e] for e in range(sd)]) for d in range(sd))
    np.testing.assert_allclose(Jc, np.kron(UPWIND, Mx), atol=1e-15)
    np.testing.assert_allclose(Jk, np.kron(mass1(dt), Kx), atol=1e-14)


# ---------------------------------------------------------------- P2 exact discrete solution
@pytest.mark.parametrize("ns,nt,spacetime", [((6, 4), 5, False), ((5, 7), 9, True), ((3, 4, 2), 4, False)])
def test_exact_discrete_solution_insulated(ns, nt, spacetime):
    """Uniform C and Q, any conductivity design, insulated sides, T = 0 at t = 0:
    T_n = n Q dt / C for n < N_t and T_N = (N_t - 1/2) Q dt / C, uniform in space."""
    C, Q = 2.0, 3.0
    mat = O.Material(C_ins=C, C_con=C, k_ins=0.1, k_con=1.0, p_c=1, p_k=3)
    m = O.Mesh(ns, nt, tau=1.3, mat=mat, bc="none")
    rng = np.random.default_rng(0)
    g = rng.random(m.elem_shape if spacetime else tuple(reversed(ns)))
    sol = O.forward(m, g, "uniform", Q)
    T = sol.s.reshape(m.node_shape)
    expect = np.array([n * Q * m.dt / C for n in range(nt)] + [(nt - 0.5) * Q * m.dt / C])
    for n in range(nt + 1):
        np.testing.assert_allclose(T[n], expect[n], rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------- P3 energy balance
def test_energy_balance_reactions():
    """Time-constant capacity: (sum of sink reactions) + (sum of f) = int C T(x, tau) dx."""
    mat = O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
    m = O.Mesh((8, 6), 7, mat=mat, bc="patch_left", bc_width=0.4)
    g = np.random.default_rng(1).random((6, 8))
    A_unc = O.assemble_unconstrained(m, g)
    sol = O.forward(m, g, "sin_t", 2.0)
    f_unc = O.assemble_source(m, O.source_fn("sin_t", 2.0), constrained=False)
    dmask = O.dirichlet_mask(m)
    R = A_unc @ sol.s - f_unc
    np.testing.assert_allclose(R[~dmask], 0.0, atol=1e-12)
    lhs = R[dmask].sum() + f_unc.sum()
    # int_Omega C(x) T_h(x, tau) dx with the bilinear interpolant of the last plane: each
    # element integrates exactly to C_e * (area / 4) * (sum of its 4 corner values).
    T = sol.s.reshape(m.node_shape)[-1]
    C = O.simp_C(mat, g)
    corner_sum = T[:-1, :-1] + T[1:, :-1] + T[:-1, 1:] + T[1:, 1:]
    rhs = np.sum(C * corner_sum) * m.h[0] * m.h[1] / 4.0
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


# ---------------------------------------------------------------- P4 Kronecker form + block elimination
@pytest.mark.parametrize("ns,nt", [((5, 4), 6), ((3, 3, 2), 3)])
def test_uniform_coefficient_kronecker_assembly_and_block_solve(ns, nt):
    mat = O.Material(C_ins=0.7, C_con=0.7, k_ins=0.2, k_con=0.2, p_c=1, p_k=1)
    m = O.Mesh(ns, nt, tau=0.8, mat=mat, bc="patch_bottom", bc_width=0.5)
    g = np.full(tuple(reversed(ns)), 0.3)
    A_unc = O.assemble_unconstrained(m, g)
    Mx, Kx = kron_spatial_mass_stiff(ns, m.h)
    J = 0.7 * sp.kron(glob_upwind(nt), Mx) + 0.2 * sp.kron(glob_mass(nt, m.dt), Kx)
    np.testing.assert_allclose(A_unc.toarray(), J.toarray(), atol=1e-14)
    A = O.assemble(m, g)
    f = O.assemble_source(m, O.source_fn("uniform", 1.0))
    x1 = O.solve_direct(A, f)
    x2 = O.solve_block_tridiag_time(A, f, nt)
    np.testing.assert_allclose(x1, x2, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- P5 manufactured solutions
def _mms_error(nx, nt, g, gp, k=0.7, C=1.3, planes=None):
    mat = O.Material(C_ins=C, C_con=C, k_ins=k, k_con=k, p_c=1, p_k=1)
    m = O.Mesh((nx, nx), nt, mat=mat, bc="all_walls")
    Q = lambda t, y, x: (C * gp(t) + 2 * k * math.pi ** 2 * g(t)) * np.sin(math.pi * x) * np.sin(math.pi * y)
    A = O.assemble(m, np.zeros((nx, nx)))
    f = O.assemble_source(m, Q, nq=4)
    s = O.solve_direct(A, f)
    t, y, x = O.node_coords(m)
    ex = g(t) * np.sin(math.pi * x) * np.sin(math.pi * y)
    err = np.abs(s - ex).reshape(m.node_shape)
    if planes is not None:
        err = err[planes(nt)]
    return err.max()


def test_manufactured_first_order_in_time():
    """Stabilised scheme: first order in time (Sec. 3.1.1)."""
    e = [_mms_error(24, nt, lambda t: t ** 2, lambda t: 2 * t) for nt in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[0] > 0.7 and 0.85 < orders[1] < 1.2, (e, orders)


def test_manufactured_time_only_first_order():
    """Spatially uniform solution T = sin(3t) on an insulated box: no spatial error, so the
    nodal error is the time error alone and halves with dt."""
    errs = []
    for nt in (16, 32, 64, 128):
        mat = O.Material(C_ins=1.7, C_con=1.7, k_ins=0.4, k_con=0.4, p_c=1, p_k=1)
        m = O.Mesh((2, 2), nt, mat=mat, bc="none")
        A = O.assemble(m, np.zeros((2, 2)))
        f = O.assemble_source(m, lambda t, y, x: 1.7 * 3 * np.cos(3 * t), nq=5)
        s = O.solve_direct(A, f)
        t = O.node_coords(m)[0]
        errs.append(np.abs(s - np.sin(3 * t)).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(0.9 < p < 1.1 for p in orders), (errs, orders)


def test_manufactured_second_order_in_space():
    """For a solution linear in time the time discretisation is exact away from the
    final plane (whose half step is felt a few planes back through the time mass),
    leaving the Q1 spatial error O(dx^2) on the first quarter of the planes."""
    e = [_mms_error(nx, 8, lambda t: t, lambda t: np.ones_like(t), planes=lambda nt: slice(0, nt // 4 + 1))
         for nx in (8, 16, 32)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(1.9 < p < 2.1 for p in orders), (e, orders)


# ---------------------------------------------------------------- P6 implicit time stepping
def test_difference_to_implicit_euler_is_first_order():
    """For a time-constant design the all-at-once solution differs from backward Euler
    with consistent mass on the same mesh by O(dt)."""
    mat = O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
    ns = (8, 8)
    g = np.random.default_rng(3).random((8, 8))
    diffs = []
    for nt in (8, 16, 32, 64):
        m = O.Mesh(ns, nt, mat=mat, bc="patch_left", bc_width=0.3)
        sol = O.forward(m, g, "uniform", 1.0)
        # backward Euler, written independently: (C-mass + dt K) T_n = C-mass T_{n-1} + dt F
        C = O.simp_C(mat, g)
        k = O.simp_k(mat, g)
        Mc = np.zeros((81, 81)); Kk = np.zeros((81, 81)); F = np.zeros(81)
        h = m.h[0]
        Me = np.kron(mass1(h), mass1(h)); Ke = np.kron(stiff1(h), mass1(h)) + np.kron(mass1(h), stiff1(h))
        for ey in range(8):
            for ex in range(8):
                idx = [(ey + a // 2) * 9 + ex + a % 2 for a in range(4)]
                Mc[np.ix_(idx, idx)] += C[ey, ex] * Me
                Kk[np.ix_(idx, idx)] += k[ey, ex] * Ke
                F[idx] += Me.sum(axis=1)
        dm = O.dirichlet_mask(m).reshape(nt + 1, 81)[1]
        T = np.zeros(81)
        traj = [T]
        Lhs = Mc + m.dt * Kk
        Lhs[dm] = 0; Lhs[:, dm] = 0; Lhs[dm, dm] = 1
        for n in range(nt):
            r = Mc @ T + m.dt * F
            r[dm] = 0
            T = np.linalg.solve(Lhs, r)
            traj.append(T)
        traj = np.array(traj)
        # the oracle's BDF1 reference solver (Sec. 4) is this scheme
        np.testing.assert_allclose(O.bdf1_forward(m, g, "uniform", 1.0), traj, rtol=0, atol=1e-13 * np.abs(traj).max())
        st = sol.s.reshape(nt + 1, 81)
        diffs.append(np.abs(st[: nt] - traj[: nt]).max())  # last plane excluded (half step)
    orders = [math.log2(diffs[i] / diffs[i + 1]) for i in range(3)]
    assert orders[-1] > 0.8 and orders[-2] > 0.7, (diffs, orders)


# ---------------------------------------------------------------- P7 brute force on tiny meshes
def _hat(x, X, h):
    return np.maximum(0.0, 1.0 - np.abs(x - X) / h)


def _dhat(x, X, h):
    inside = np.abs(x - X) < h
    return np.where(inside, -np.sign(x - X) / h, 0.0)


def _bruteforce_J(ns, nt, tau, mat, ge):
    """a(N_j, N_i) by integrating global hat functions cell by cell (3-point Gauss),
    without element connectivity or local numbering."""
    nx, ny = ns
    hx, hy, dt = 1.0 / nx, 1.0 / ny, tau / nt
    nodes = [(n, j, i) for n in range(nt + 1) for j in range(ny + 1) for i in range(nx + 1)]
    N = len(nodes)
    X = np.array([[i * hx, j * hy, n * dt] for (n, j, i) in nodes])
    gp, gw = O.gauss_1d(3)
    J = np.zeros((N, N))
    for en in range(nt):
        for ey in range(ny):
            for ex in range(nx):
                C = O.simp_C(mat, ge[en, ey, ex]); k = O.simp_k(mat, ge[en, ey, ex])
                for a in range(3):
                    for b in range(3):
                        for c in range(3):
                            x = (ex + gp[a]) * hx; y = (ey + gp[b]) * hy; t = (en + gp[c]) * dt
                            w = gw[a] * gw[b] * gw[c] * hx * hy * dt
                            hxv = _hat(x, X[:, 0], hx); hyv = _hat(y, X[:, 1], hy); htv = _hat(t, X[:, 2], dt)
                            Nv = hxv * hyv * htv
                            Nx = _dhat(x, X[:, 0], hx) * hyv * htv
                            Ny = hxv * _dhat(y, X[:, 1], hy) * htv
                            Nt = hxv * hyv * _dhat(t, X[:, 2], dt)
                            J += w * (C * np.outer(Nv, Nt) + 0.5 * C * dt * np.outer(Nt, Nt)
                                      + k * (np.outer(Nx, Nx) + np.outer(Ny, Ny)))
    return J


def test_bruteforce_assembly_and_dense_solves():
    mat = O.Material()
    ns, nt = (2, 3), 2
    m = O.Mesh(ns, nt, tau=0.7, mat=mat, bc="patch_left", bc_width=0.4)
    ge = np.random.default_rng(5).random(m.elem_shape)
    Jb = _bruteforce_J(ns, nt, 0.7, mat, ge)
    A_unc = O.assemble_unconstrained(m, ge).toarray()
    np.testing.assert_allclose(A_unc, Jb, atol=1e-13)
    # constrained dense solve and dense adjoint versus the oracle's sparse direct solves
    dm = O.dirichlet_mask(m)
    Jd = Jb.copy(); Jd[dm] = 0; Jd[:, dm] = 0; Jd[dm, dm] = 1
    f = O.assemble_source(m, O.source_fn("uniform", 1.0))
    sol = O.forward(m, ge, "uniform", 1.0)
    np.testing.assert_allclose(sol.s, np.linalg.solve(Jd, f), rtol=1e-12, atol=1e-14)
    lam = O.adjoint(sol.A, f, dm, sol.lu)
    np.testing.assert_allclose(lam, np.linalg.solve(Jd.T, f), rtol=1e-12, atol=1e-14)
    # the patch on x = 0 with width 0.4 of a 3-element edge holds node j iff |2j - 3| <= 1.2
    T = dm.reshape(m.node_shape)
    assert T[0].all() and T[1:, 1, 0].all() and T[1:, 2, 0].all()
    assert not T[1:, 0, 0].any() and not T[1:, 3, 0].any() and not T[1:, :, 1:].any()


def test_patch_node_counts():
    """Left-edge patch of width L/10: nodes 15..17 on a 32-element edge, 25 nodes at 256."""
    for n, cnt in ((32, 3), (256, 25), (64, 7)):
        m = O.Mesh((n, n), 1, bc="patch_left")
        T = O.dirichlet_mask(m).reshape(m.node_shape)[1]
        assert T.sum() == cnt and T[:, 0].sum() == cnt
    m = O.Mesh((64, 64, 64), 1, bc="patch_left")
    assert O.dirichlet_mask(m).reshape(m.node_shape)[1].sum() == 49


# ---------------------------------------------------------------- P8 Algorithm 1 versus the paper
def _read_golden_hierarchies():
    rows = []
    with open(os.path.join(GOLDEN, "paper_hierarchies.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            case, tau, matl, levels = [p.strip() for p in line.split("|")]
            Ci, Cc, ki, kc = map(float, matl.split())
            lev = [tuple(map(int, L.split("x"))) for L in levels.split()]
            rows.append((case, float(tau), O.Material(Ci, Cc, ki, kc), lev))
    return rows


@pytest.mark.parametrize("case,tau,mat,levels", _read_golden_hierarchies())
def test_algorithm1_reproduces_paper_tables(case, tau, mat, levels):
    m = O.Mesh((640, 640), 1280, tau=tau, mat=mat)
    got = O.hierarchy(m, lam_crit=0.5, n_levels=len(levels))
    assert [(l.ns[0], l.ns[1], l.nt) for l in got] == levels


def test_dof_counts_match_paper():
    with open(os.path.join(GOLDEN, "paper_dof_counts.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            mesh, dofs, _ = [p.strip() for p in line.split("|")]
            dims = list(map(int, mesh.split("x")))
            if len(dims) == 3:
                m = O.Mesh((dims[0], dims[1]), dims[2])
                assert m.n_nodes == int(dofs)
            else:
                assert (dims[0] + 1) * (dims[1] + 1) == int(dofs)


# ---------------------------------------------------------------- transfers and P9 Galerkin
def test_prolongation_reproduces_affine_functions():
    for fine, coarse in (((8, 6), 4), ((8, 6), 2)):
        mf = O.Mesh(fine, 4)
        levels = O.hierarchy(mf, n_levels=2)
        L0 = O.Level((8, 6), 4, mf.h, mf.dt)
        L1 = O.Level((4, 3), 4, tuple(2 * x for x in mf.h), mf.dt) if coarse == 4 else \
            O.Level((8, 6), 2, mf.h, 2 * mf.dt)
        P = O.prolongation(L0, L1)
        aff = lambda t, y, x: 0.3 + 1.7 * x - 0.9 * y + 2.1 * t
        cm = O.Mesh(L1.ns, L1.nt, tau=L1.dt * L1.nt)
        fm = O.Mesh(L0.ns, L0.nt, tau=L0.dt * L0.nt)
        np.testing.assert_allclose(P @ aff(*O.node_coords(cm)), aff(*O.node_coords(fm)), atol=1e-13)


def _interior_rows(m, margin=2):
    idx = np.indices(m.node_shape).reshape(len(m.node_shape), -1)
    ok = np.ones(idx.shape[1], dtype=bool)
    for ax, n in enumerate(m.node_shape):
        ok &= (idx[ax] >= margin) & (idx[ax] <= n - 1 - margin)
    return np.nonzero(ok)[0]


@pytest.mark.parametrize("kind", ["space", "time"])
def test_galerkin_equals_rediscretisation_for_uniform_coefficients(kind):
    """Uniform coefficients: on interior rows P^T J P is the coarse Q1 operator; for time
    coarsening its stabilising diffusion keeps the fine dt (k_ad = C dt_fine / 2)."""
    C, k = 0.8, 0.35
    mat = O.Material(C_ins=C, C_con=C, k_ins=k, k_con=k, p_c=1, p_k=1)
    mf = O.Mesh((8, 8), 8, mat=mat, bc="none")
    L0 = O.Level(mf.ns, mf.nt, mf.h, mf.dt)
    if kind == "space":
        L1 = O.Level((4, 4), 8, tuple(2 * x for x in mf.h), mf.dt)
    else:
        L1 = O.Level((8, 8), 4, mf.h, 2 * mf.dt)
    mg = O.build_mg(mf, np.zeros((8, 8)), [L0, L1])
    Ac = mg[1].A
    mc = O.Mesh(L1.ns, L1.nt, tau=1.0, mat=mat, bc="none")
    Mx, Kx = kron_spatial_mass_stiff(L1.ns, L1.h)
    dt_c = L1.dt
    # coarse time factors written from the 1D integrals on a 2 dt_f slab with k_ad = C dt_f / 2
    Dt_el = np.array([[-0.5, 0.5], [-0.5, 0.5]]) + 0.5 * mf.dt / dt_c * np.array([[1.0, -1.0], [-1.0, 1.0]])
    nt = L1.nt
    Dg = sp.lil_matrix((nt + 1, nt + 1))
    for s in range(nt):
        for a in range(2):
            for b in range(2):
                Dg[s + a, s + b] += Dt_el[a, b]
    Jc = C * sp.kron(Dg.tocsr(), Mx) + k * sp.kron(glob_mass(nt, dt_c), Kx)
    rows = _interior_rows(mc)
    np.testing.assert_allclose(Ac[rows].toarray(), Jc.tocsr()[rows].toarray(), atol=1e-13)


# ---------------------------------------------------------------- adjoint and gradients
def test_adjoint_duality():
    m = O.Mesh((6, 5), 6, mat=O.Material(), bc="patch_left", bc_width=0.4)
    g = np.random.default_rng(7).random((5, 6))
    sol = O.forward(m, g, "uniform", 1.0)
    dm = O.dirichlet_mask(m)
    rng = np.random.default_rng(8)
    c = rng.standard_normal(m.n_nodes); c[dm] = 0
    lam = O.adjoint(sol.A, c, dm, sol.lu)
    # c^T s = Lambda^T f for a linear functional of the state
    np.testing.assert_allclose(c @ sol.s, lam @ sol.f, rtol=1e-12)


@pytest.mark.parametrize("spacetime", [False, True])
def test_compliance_gradient_complex_step_and_fd(spacetime):
    mat = O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
    m = O.Mesh((4, 4), 4, mat=mat, bc="patch_left", bc_width=0.5)
    rng = np.random.default_rng(11)
    g = 0.2 + 0.6 * rng.random(m.elem_shape if spacetime else (4, 4))
    sol = O.forward(m, g, "sin_t", 1.0)
    dm = O.dirichlet_mask(m)
    lam = O.adjoint(sol.A, sol.f, dm, sol.lu)
    grad = O.sensitivities(m, g, sol.s, lam, extruded=not spacetime)
    for flat in rng.choice(g.size, 5, replace=False):
        idx = np.unravel_index(flat, g.shape)
        gc = g.astype(complex)
        gc[idx] += 1e-30j
        A = O.assemble(m, gc)
        s = O.solve_direct(A, sol.f.astype(complex))
        cs = np.imag(sol.f @ s) / 1e-30
        np.testing.assert_allclose(grad[idx], cs, rtol=1e-10)
        gp, gm = g.copy(), g.copy()
        gp[idx] += 1e-6; gm[idx] -= 1e-6
        fd = (O.forward(m, gp, "sin_t", 1.0).s @ sol.f - O.forward(m, gm, "sin_t", 1.0).s @ sol.f) / 2e-6
        np.testing.assert_allclose(grad[idx], fd, rtol=1e-6)


def test_pnorm_value_and_gradient():
    m = O.Mesh((3, 3), 3, bc="none")
    s = np.random.default_rng(2).random(m.n_nodes)
    P = 20
    phi, g = O.pnorm(m, s, P)
    # value from the definition, element by element with explicit loops
    T = s.reshape(m.node_shape)
    acc = 0.0
    for n in range(3):
        for j in range(3):
            for i in range(3):
                acc += T[n:n + 2, j:j + 2, i:i + 2].mean() ** P
    np.testing.assert_allclose(phi, acc ** (1.0 / P), rtol=1e-13)
    for k in (0, 17, 40, 63):
        e = np.zeros_like(s); e[k] = 1e-4
        fd = (O.pnorm(m, s + e, P)[0] - O.pnorm(m, s - e, P)[0]) / 2e-4
        np.testing.assert_allclose(g[k], fd, rtol=1e-5, atol=1e-9 * np.abs(g).max())


# ---------------------------------------------------------------- source quadrature reading
def test_source_quadrature_two_point_gauss_error_is_third_order():
    """2-point Gauss on a slab of width dt errs by dt^5 f^(4) / 4320 with f = N_a q; since
    N_a' = O(1/dt) the nodal load error relative to the nodal measure is O(dt^3)."""
    errs = []
    for nt in (32, 64, 128):
        m = O.Mesh((2, 2), nt, bc="none")
        f2 = O.assemble_source(m, O.source_fn("sin_t", 1.0), nq=2, constrained=False)
        f6 = O.assemble_source(m, O.source_fn("sin_t", 1.0), nq=6, constrained=False)
        errs.append(np.abs(f2 - f6).max() / (m.dt * m.h[0] * m.h[1]))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.8 < p < 3.2 for p in orders), (errs, orders)


def test_uniform_source_is_integral_of_hat_functions():
    m = O.Mesh((4, 3), 5, tau=2.0, bc="none")
    f = O.assemble_source(m, O.source_fn("uniform", 2.5), constrained=False).reshape(m.node_shape)
    wx = np.full(5, m.h[0]); wx[[0, -1]] /= 2
    wy = np.full(4, m.h[1]); wy[[0, -1]] /= 2
    wt = np.full(6, m.dt); wt[[0, -1]] /= 2
    np.testing.assert_allclose(f, 2.5 * wt[:, None, None] * wy[None, :, None] * wx[None, None, :], rtol=1e-13)


# ---------------------------------------------------------------- smoother and V-cycle
def test_gmres_smoother_minimises_residual_over_krylov_space():
    m = O.Mesh((6, 6), 6, mat=O.Material(), bc="patch_left", bc_width=0.4)
    g = np.random.default_rng(4).random((6, 6))
    A = O.assemble(m, g)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(m.n_nodes); b[O.dirichlet_mask(m)] = 0
    x0 = rng.standard_normal(m.n_nodes) * 0.1
    x = O.gmres_jacobi(A, b, x0, 10)
    dinv = 1.0 / A.diagonal()
    r0 = b - A @ x0
    K = [r0]
    for _ in range(9):
        K.append(A @ (dinv * K[-1]))
    K = np.array(K).T
    K, _ = np.linalg.qr(K)
    y = np.linalg.lstsq(A @ (dinv[:, None] * K), r0, rcond=None)[0]
    xb = x0 + dinv * (K @ y)
    np.testing.assert_allclose(np.linalg.norm(b - A @ x), np.linalg.norm(b - A @ xb), rtol=1e-8)
    np.testing.assert_allclose(x, xb, rtol=1e-6, atol=1e-8 * np.abs(xb).max())


def test_vcycle_is_a_contraction_and_exact_on_one_level():
    mat = O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)
    m = O.Mesh((16, 16), 16, mat=mat)
    g = np.random.default_rng(6).random((16, 16))
    levels = O.hierarchy(m, coarse_cap=400)
    assert len(levels) >= 3
    mg = O.build_mg(m, g, levels)
    f = O.assemble_source(m, O.source_fn("uniform"))
    x = np.zeros_like(f)
    res = [np.linalg.norm(f)]
    for _ in range(4):
        x = x + O.vcycle(mg, f - mg[0].A @ x)
        res.append(np.linalg.norm(f - mg[0].A @ x))
    assert all(res[i + 1] < 0.5 * res[i] for i in range(4)), res
    one = O.build_mg(m, g, levels[:1])
    np.testing.assert_allclose(O.vcycle(one, f), O.solve_direct(mg[0].A, f), rtol=1e-10, atol=1e-14)
    # coarse prescribed sets are the geometric rule evaluated on the coarse grids
    for l in range(1, len(levels)):
        L = levels[l]
        cm = O.Mesh(L.ns, L.nt, mat=mat)
        np.testing.assert_array_equal(mg[l].mask, O.dirichlet_mask(cm))


def test_sin_source_moments_match_closed_form():
    """q(t) = 1 + 0.5 sin(2 pi 4 t) on [0, 1]: sum_i f_i = |Omega| int q dt = 1 and, since the
    hat functions interpolate t exactly, sum_i t_i f_i = int t q dt = 1/2 - 1/(16 pi)."""
    m = O.Mesh((3, 2), 64, bc="none")
    f = O.assemble_source(m, O.source_fn("sin_t", 1.0), nq=6, constrained=False)
    t = O.node_coords(m)[0]
    np.testing.assert_allclose(f.sum(), 1.0, rtol=1e-12)
    np.testing.assert_allclose(t @ f, 0.5 - 1.0 / (16.0 * math.pi), rtol=1e-10)
    f2 = O.assemble_source(m, O.source_fn("sin_t", 1.0), nq=2, constrained=False)
    np.testing.assert_allclose(t @ f2, 0.5 - 1.0 / (16.0 * math.pi), rtol=1e-5)


def test_apply_rows_matches_assembled_operator():
    """Row-by-row evaluation (used for sampled checks on large meshes) equals the assembled
    constrained operator, for space-time and extruded designs in 2+1D and 3+1D."""
    rng = np.random.default_rng(12)
    for ns, nt, st in (((5, 4), 6, True), ((5, 4), 3, False), ((3, 2, 2), 3, False)):
        m = O.Mesh(ns, nt, mat=O.Material(), bc="patch_bottom", bc_width=0.6)
        g = rng.random(m.elem_shape if st else tuple(reversed(ns)))
        A = O.assemble(m, g)
        x = rng.random(m.n_nodes)
        rows = np.arange(m.n_nodes)
        np.testing.assert_allclose(O.apply_rows(m, g, x, rows), A @ x, rtol=1e-13, atol=1e-15)
        xs = x - 0.5  # both signs
        np.testing.assert_allclose(O.apply_rows(m, g, xs, rows, absolute=True),
                                   O.abs_operator(m, g) @ np.abs(xs), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("ns,nt,kind", [((5, 4), 6, "sin_t"), ((3, 2, 4), 3, "uniform")])
def test_source_rows_match_assembled_source(ns, nt, kind):
    """The row-by-row source (used where the mesh is too large to assemble) equals the
    assembled source vector on every node."""
    m = O.Mesh(ns, nt, bc="patch_left", bc_width=0.5)
    Q = O.source_fn(kind, 1.0, 1.0, 0.5, 4.0)
    f = O.assemble_source(m, Q)
    rows = np.arange(m.n_nodes)
    np.testing.assert_allclose(O.source_rows(m, Q, rows), f, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------- V-cycle structure (Sec. 3.2)
def _minres_smooth(A, b, x0, m):
    """Independent statement of m GMRES steps with right Jacobi preconditioning: the x0 + D^-1 K y
    of least residual norm over the Krylov space K = span{r0, (A D^-1) r0, ..., (A D^-1)^(m-1) r0}
    (dense, power basis orthonormalised by a QR factorisation, then numpy least squares)."""
    A = np.asarray(A.toarray() if sp.issparse(A) else A)
    dinv = 1.0 / np.diag(A)
    r0 = b - A @ x0
    K = [r0]
    for _ in range(m - 1):
        K.append(A @ (dinv * K[-1]))
    Q, _ = np.linalg.qr(np.array(K).T)
    y = np.linalg.lstsq(A @ (dinv[:, None] * Q), r0, rcond=None)[0]
    return x0 + dinv * (Q @ y)


def _two_level_hand(A, Ac, Pt, b, m):
    """The two-level cycle written out step by step from Sec. 3.2: pre-smoothing from zero,
    residual, restriction by Pt^T, exact coarse solve, prolongation by Pt, post-smoothing from
    the corrected iterate."""
    A = A.toarray()
    x = _minres_smooth(A, b, np.zeros_like(b), m)
    r = b - A @ x
    ec = np.linalg.solve(Ac.toarray(), Pt.toarray().T @ r)
    x = x + Pt.toarray() @ ec
    return _minres_smooth(A, b, x, m)


@pytest.mark.parametrize("transpose", [False, True])
def test_vcycle_two_level_equals_hand_composition(transpose):
    """A two-level V-cycle on a 4x4x4 mesh equals the cycle composed by hand from an
    independently computed minimal-residual smoother.  Post-smoothing started from zero
    instead of the corrected iterate, a missing post-smoothing, a sign error in the coarse
    correction, or an adjoint cycle that transposes only the fine level all change the result
    far beyond the tolerance (each was planted in a copy of the cycle and fails here)."""
    mat = O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)
    m = O.Mesh((4, 4), 4, mat=mat, bc="patch_left", bc_width=0.5)
    g = np.random.default_rng(21).random((4, 4))
    levels = O.hierarchy(m, n_levels=2)
    assert len(levels) == 2
    mg = O.build_mg(m, g, levels)
    b = np.random.default_rng(22).standard_normal(m.n_nodes)
    b[mg[0].mask] = 0
    A = mg[0].A.T.tocsr() if transpose else mg[0].A
    Ac = mg[1].A.T.tocsr() if transpose else mg[1].A
    for nsm, tol in ((2, 1e-11), (3, 1e-10)):
        ref = _two_level_hand(A, Ac, mg[0].Pt, b, nsm)
        got = O.vcycle(mg, b, nsmooth=nsm, transpose=transpose)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), nsm
    # the transposed cycle differs from the forward one (the operator is not symmetric)
    if transpose:
        fwd = O.vcycle(mg, b, nsmooth=2)
        assert np.abs(fwd - O.vcycle(mg, b, nsmooth=2, transpose=True)).max() > 1e-6 * np.abs(fwd).max()


def test_vcycle_transposed_one_level_is_the_transposed_solve():
    """On a one-level hierarchy the transposed V-cycle is the coarsest solve with A^T."""
    m = O.Mesh((5, 4), 6, mat=O.Material(), bc="patch_bottom", bc_width=0.4)
    g = np.random.default_rng(23).random((4, 5))
    one = O.build_mg(m, g, O.hierarchy(m)[:1])
    b = np.random.default_rng(24).standard_normal(m.n_nodes)
    A = one[0].A
    ref = np.linalg.solve(A.toarray().T, b)
    np.testing.assert_allclose(O.vcycle(one, b, transpose=True), ref, rtol=1e-10, atol=1e-13 * np.abs(ref).max())
    assert np.abs(O.vcycle(one, b) - ref).max() > 1e-6 * np.abs(ref).max()


def test_transposed_vcycle_contracts_on_the_transposed_operator():
    """Preconditioned Richardson with the transposed cycle converges on A^T lambda = b (the
    adjoint system of Sec. 3.3.3): at least 2x residual reduction per cycle."""
    mat = O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)
    m = O.Mesh((16, 16), 16, mat=mat)
    g = np.random.default_rng(6).random((16, 16))
    mg = O.build_mg(m, g, O.hierarchy(m, coarse_cap=400))
    At = mg[0].A.T.tocsr()
    b = O.assemble_source(m, O.source_fn("uniform"))
    x = np.zeros_like(b)
    res = [np.linalg.norm(b)]
    for _ in range(4):
        x = x + O.vcycle(mg, b - At @ x, transpose=True)
        res.append(np.linalg.norm(b - At @ x))
    assert all(res[i + 1] < 0.5 * res[i] for i in range(4)), res


# ---------------------------------------------------------------- single-precision runs
def test_float32_smoother_runs_in_single_precision_and_tracks_float64():
    """The float32 variant of the smoother returns float32 values that differ from the
    float64 run by more than float64 rounding (so it really computes in single precision)
    but by no more than a few hundred float32 unit roundoffs (so it is the same algorithm)."""
    m = O.Mesh((6, 6), 6, mat=O.Material(), bc="patch_left", bc_width=0.4)
    A = O.assemble(m, np.random.default_rng(4).random((6, 6)))
    rng = np.random.default_rng(9)
    b = rng.standard_normal(m.n_nodes); b[O.dirichlet_mask(m)] = 0
    x0 = rng.standard_normal(m.n_nodes) * 0.1
    x64 = O.gmres_jacobi(A, b, x0, 6)
    x32 = O.gmres_jacobi(A, b, x0, 6, dtype=np.float32)
    assert x32.dtype == np.float32
    err = np.abs(x32.astype(np.float64) - x64).max() / np.abs(x64).max()
    assert 1e-10 < err < 300 * 2.0 ** -24, err
    # the single-precision V-cycle keeps the same structure and contracts as well
    mat = O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)
    mm = O.Mesh((16, 16), 16, mat=mat)
    mg = O.build_mg(mm, np.random.default_rng(6).random((16, 16)), O.hierarchy(mm, coarse_cap=400))
    f = O.assemble_source(mm, O.source_fn("uniform"))
    v64 = O.vcycle(mg, f)
    v32 = O.vcycle(mg, f, dtype=np.float32)
    assert v32.dtype == np.float32
    e = np.abs(v32.astype(np.float64) - v64).max() / np.abs(v64).max()
    assert 1e-10 < e < 1e-3, e
    r0 = np.linalg.norm(f)
    assert np.linalg.norm(f - mg[0].A @ v32.astype(np.float64)) < 0.5 * r0


def test_abs_operator_bounds_the_operator_and_is_exact_on_one_element():
    """|J|_elem >= |J| entry by entry, with equality on one element when only the capacity part
    or only the conductivity part is present (nothing is summed), and it bounds the float32
    evaluation error of the element-by-element product."""
    mat = O.Material()
    g1 = np.array([[0.37]])
    for part in (O.Material(C_ins=0.5, C_con=1.0, k_ins=0.0, k_con=0.0), O.Material(C_ins=0.0, C_con=0.0)):
        one = O.Mesh((1, 1), 1, mat=part, bc="none", ext=(0.3, 0.7))
        np.testing.assert_allclose(O.abs_operator(one, g1).toarray(), np.abs(O.assemble(one, g1).toarray()),
                                   rtol=1e-15, atol=0)
    m = O.Mesh((5, 4), 3, mat=mat, bc="patch_left", bc_width=0.5)
    g = np.random.default_rng(25).random((3, 4, 5))
    A = O.assemble(m, g).toarray()
    B = O.abs_operator(m, g).toarray()
    assert np.all(B >= np.abs(A) - 1e-15 * np.abs(A).max())
    assert (B > np.abs(A) + 1e-12 * np.abs(A).max()).any()  # cancellation exists between elements
    # a float32 element-by-element product stays within 16 u32 |J|_elem |x| per row
    x = np.random.default_rng(26).standard_normal(m.n_nodes)
    ge = O.element_gamma(m, g)
    Jc, Jk = O.element_matrices(m.h, m.dt)
    conn = O.element_connectivity(m)
    dm = O.dirichlet_mask(m)
    xm = np.where(dm, 0.0, x).astype(np.float32)
    y = np.zeros(m.n_nodes, dtype=np.float32)
    Cs = O.simp_C(mat, ge).astype(np.float32)
    ks = O.simp_k(mat, ge).astype(np.float32)
    for e in range(m.n_elem):
        Ee = Cs[e] * Jc.astype(np.float32) + ks[e] * Jk.astype(np.float32)
        np.add.at(y, conn[e], (Ee @ xm[conn[e]]).astype(np.float32))
    y = np.where(dm, x.astype(np.float32), y).astype(np.float64)
    err = np.abs(y - A @ x)
    assert np.all(err <= 16 * 2.0 ** -24 * (B @ np.abs(x)) + 1e-30)


# ---------------------------------------------------------------- PDE filter and projection (Sec. 3.3.2)
def _cosine_mode(m, k):
    """Nodal field prod_d cos(k_d pi i_d / n_d) in node order (t, [z,] y, x); k = (kx, ky, [kz,] kt)."""
    axes_n = [m.nt] + list(reversed(m.ns))
    axes_k = [k[-1]] + list(reversed(k[:-1]))
    grids = [np.cos(kk * np.pi * np.arange(n + 1) / n) for kk, n in zip(axes_k, axes_n)]
    out = grids[0]
    for gg in grids[1:]:
        out = np.multiply.outer(out, gg)
    return out.reshape(-1)


def _boundary_weights(m):
    axes_n = [m.nt] + list(reversed(m.ns))
    ws = []
    for n in axes_n:
        w = np.ones(n + 1); w[0] = w[-1] = 0.5
        ws.append(w)
    out = ws[0]
    for w in ws[1:]:
        out = np.multiply.outer(out, w)
    return out.reshape(-1)


@pytest.mark.parametrize("ns,nt", [((5, 4), 6), ((3, 4, 2), 3)])
def test_filter_operator_acts_on_cosine_modes_by_its_closed_form(ns, nt):
    """On a regular Q1 mesh with natural boundary conditions, sampled cosines are eigenvectors of the
    1-D mass and stiffness matrices up to halved boundary rows: M v = mu (w v), K v = kappa (w v) with
    mu = h (4 + 2 cos theta) / 6, kappa = (2 - 2 cos theta) / h, theta = k pi / n.  So the filter matrix
    acts on prod_d cos(k_d pi x_d / L_d) by
    sigma = prod mu + (r_x^2/12) sum_spatial kappa_a prod_{d != a} mu_d + (r_t^2/12) kappa_t prod_{d != t} mu_d."""
    ext = tuple(0.6 + 0.2 * d for d in range(len(ns)))
    m = O.Mesh(ns, nt, ext=ext, tau=0.9, bc="none")
    r_x, r_t = 0.31, 0.23
    A = O.filter_operator(m, r_x, r_t)
    w = _boundary_weights(m)
    sizes = list(m.h) + [m.dt]
    counts = list(ns) + [nt]
    for k in itertools.product(*[range(0, c + 1, max(1, c // 2)) for c in counts]):
        mu = [hh * (4 + 2 * np.cos(kk * np.pi / c)) / 6 for hh, kk, c in zip(sizes, k, counts)]
        ka = [(2 - 2 * np.cos(kk * np.pi / c)) / hh for hh, kk, c in zip(sizes, k, counts)]
        sd = len(ns)
        sigma = np.prod(mu)
        for a in range(sd + 1):
            coef = (r_x if a < sd else r_t) ** 2 / 12.0
            sigma += coef * ka[a] * np.prod([mu[d] for d in range(sd + 1) if d != a])
        psi = _cosine_mode(m, k)
        np.testing.assert_allclose(A @ psi, sigma * w * psi, rtol=0, atol=1e-13 * np.abs(sigma))


def test_filter_preserves_constants_and_volume_and_is_symmetric():
    m = O.Mesh((6, 5), 4, ext=(1.0, 0.8), tau=1.2, bc="none")
    rng = np.random.default_rng(31)
    g = rng.random(m.elem_shape)
    r_x, r_t = 2.4 * m.h[0], 2.4 * m.dt
    np.testing.assert_allclose(O.pde_filter(m, np.ones(m.elem_shape), r_x, r_t), 1.0, rtol=1e-13)
    gt = O.pde_filter(m, g, r_x, r_t)
    np.testing.assert_allclose(gt.sum(), g.sum(), rtol=1e-13)  # equal element volumes
    assert np.abs(gt - g).max() > 1e-3 and gt.min() >= 0 and gt.max() <= 1
    a, b = rng.standard_normal(m.elem_shape), rng.standard_normal(m.elem_shape)
    np.testing.assert_allclose(np.sum(a * O.pde_filter(m, b, r_x, r_t)), np.sum(b * O.pde_filter(m, a, r_x, r_t)),
                               rtol=1e-12)


def test_filter_of_an_extruded_design_is_time_constant():
    """A time-constant design filtered on the full space-time mesh gives the same value on every slab,
    equal to the one-slab (spatial) filter used for extruded designs."""
    m = O.Mesh((5, 4), 6, bc="none")
    g2 = np.random.default_rng(32).random((4, 5))
    r_x, r_t = 0.5, 0.4
    full = O.pde_filter(m, np.broadcast_to(g2[None], m.elem_shape).copy(), r_x, r_t)
    one = O.pde_filter(m, g2, r_x, r_t)
    for n in range(m.nt):
        np.testing.assert_allclose(full[n], one, rtol=1e-12)


def test_heaviside_projection_values_and_derivative():
    x = np.linspace(0.0, 1.0, 21)
    for beta, eta in ((32.0, 0.5), (8.0, 0.3)):
        H = O.heaviside(x, beta, eta)
        np.testing.assert_allclose(H[[0, -1]], [0.0, 1.0], atol=1e-15)
        assert np.all(np.diff(H) > 0)
        h = 1e-6
        fd = (O.heaviside(x + h, beta, eta) - O.heaviside(x - h, beta, eta)) / (2 * h)
        np.testing.assert_allclose(O.heaviside_derivative(x, beta, eta), fd, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(O.heaviside(np.array([0.5]), 32.0, 0.5), [0.5], atol=1e-15)


@pytest.mark.parametrize("spacetime", [False, True])
def test_filtered_projected_compliance_gradient_matches_central_differences(spacetime):
    """phi(gamma) = compliance of the design H(F gamma): the chain rule F (H' * dphi/dgamma_bar) with
    the adjoint sensitivities equals central differences of the whole chain."""
    m = O.Mesh((4, 4), 4, mat=O.Material(), bc="patch_left", bc_width=0.5)
    rng = np.random.default_rng(33)
    g = 0.3 + 0.4 * rng.random(m.elem_shape if spacetime else (4, 4))
    r_x, r_t, beta, eta = 0.5, 0.5, 8.0, 0.5

    def phi(gam):
        gb, _ = O.design_chain(m, gam, r_x, r_t, beta, eta)
        sol = O.forward(m, gb, "uniform", 1.0)
        return O.compliance(sol.f, sol.s), sol, gb

    p0, sol, gb = phi(g)
    _, gt = O.design_chain(m, g, r_x, r_t, beta, eta)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(m), sol.lu)
    dphys = O.sensitivities(m, gb, sol.s, lam, extruded=not spacetime)
    grad = O.chain_rule(m, dphys, gt, r_x, r_t, beta, eta)
    h = 1e-6
    for flat in rng.choice(g.size, 5, replace=False):
        idx = np.unravel_index(flat, g.shape)
        gp, gm_ = g.copy(), g.copy()
        gp[idx] += h
        gm_[idx] -= h
        fd = (phi(gp)[0] - phi(gm_)[0]) / (2 * h)
        np.testing.assert_allclose(grad[idx], fd, rtol=2e-6, atol=1e-10 * abs(p0))


# ---------------------------------------------------------------------------------------------
# Example 2's moving Gaussian source (Sec. 2.3.2)

def _ex2_source():
    # the paper's parameters: peak 1, width 0.05, radius 0.25, angular frequency pi, L = 1
    return O.source_fn("gaussian", 1.0, 0.05, 0.25, math.pi, center=(0.5, 0.5))


def test_gaussian_source_integral_is_the_closed_form():
    """The assembled (unconstrained) source sums to int int Q dx dt = q0 2 pi sigma^2 tau: the walls
    lie five widths from the circle, so the Gaussian's tail beyond them is below 1e-6 of it; a
    wrong normalisation (sigma for sigma^2, a missing 2) or peak fails by a factor."""
    om = O.Mesh((48, 48), 12, mat=O.Material(), bc="all_walls", bc_width=0.1, tau=6.0)
    f = O.assemble_source(om, _ex2_source(), nq=2, constrained=False)
    exact = 1.0 * 2.0 * math.pi * 0.05 ** 2 * 6.0
    assert abs(f.sum() / exact - 1.0) < 1e-6


def test_gaussian_source_path_and_diameter():
    """The paper's statements: the source starts at (L/2, 3L/4); one rotation takes 2 units of
    time (omega = pi); its diameter is about 0.3 (at 0.15 from the centre it is near 1 % of the
    peak).  The centroid of the assembled source on a time plane (a symmetric hat in time) sits at
    the centre of that time: (0.5, 0.75) at t = 0 and t = 2, and, moving counter-clockwise from
    the top, (0.25, 0.5) at t = 0.5 and (0.5, 0.25) at t = 1 (a swapped x / y axis in the
    quadrature would mirror these)."""
    Q = _ex2_source()
    t0 = np.zeros(1)
    assert abs(Q(t0, np.array([0.75]), np.array([0.5]))[0] - 1.0) < 1e-15
    peak_ratio = Q(t0, np.array([0.75]), np.array([0.5 + 0.15]))[0]
    assert 0.005 < peak_ratio < 0.02
    ys, xs = np.meshgrid(np.linspace(0, 1, 41), np.linspace(0, 1, 41), indexing="ij")
    assert np.allclose(Q(np.full(ys.shape, 2.0), ys, xs), Q(np.zeros(ys.shape), ys, xs), atol=1e-12)
    om = O.Mesh((64, 64), 64, mat=O.Material(), bc="all_walls", bc_width=0.1, tau=4.0)
    f = O.assemble_source(om, Q, nq=2, constrained=False).reshape(om.node_shape)
    y, x = np.meshgrid(np.linspace(0, 1, 65), np.linspace(0, 1, 65), indexing="ij")
    for n, (cx, cy) in [(8, (0.25, 0.5)), (16, (0.5, 0.25)), (24, (0.75, 0.5)), (32, (0.5, 0.75))]:
        w = f[n] / f[n].sum()
        assert abs((w * x).sum() - cx) < 2e-3 and abs((w * y).sum() - cy) < 2e-3, (n, (w * x).sum(), (w * y).sum())


# ---------------------------------------------------------------------------------------------
# Method of Moving Asymptotes (Sec. 3.3.3), one constraint

def _mma_problem(seed=0, n=400):
    rng = np.random.default_rng(seed)
    return rng.random(n) + 0.1, 0.3


def test_mma_converges_to_the_closed_form_optimum():
    """min sum c_j / x_j  s.t.  mean(x) <= V,  1e-3 <= x <= 1: convex and separable, with the
    optimum x_j = V n sqrt(c_j) / sum_k sqrt(c_k) (Lagrange; all inside the bounds here).  Forty
    MMA iterations from x = V reach it to 1e-12; a wrong sign in either approximation term, a
    swapped asymptote or a wrong root of the dual does not converge to it."""
    c, V = _mma_problem()
    n = c.size
    x = np.full(n, V)
    xo1, xo2, low, upp = x.copy(), x.copy(), x.copy(), x.copy()
    for it in range(1, 41):
        f0 = np.sum(c / x)
        x_new, low, upp, lam = O.mma_update(it, x, xo1, xo2, low, upp, -c / x ** 2 / f0, x.mean() / V - 1.0,
                                            np.full(n, 1.0 / (n * V)), xmin=1e-3, xmax=1.0)
        xo2, xo1, x = xo1, x, x_new
    exact = V * n * np.sqrt(c) / np.sqrt(c).sum()
    assert np.abs(x - exact).max() < 1e-12
    assert lam > 0 and abs(x.mean() / V - 1.0) < 1e-12


def test_mma_subproblem_solution_satisfies_its_kkt_conditions():
    """At the returned point: every free x_j is stationary for P / (U - x) + Q / (x - L); at a bound
    the derivative points outward; the multiplier is positive only where the approximated
    constraint is active (complementary slackness), and then it holds with equality."""
    rng = np.random.default_rng(3)
    n = 2000
    x = rng.uniform(0.1, 0.9, n)
    low, upp = O.mma_asymptotes(3, x, x - 0.02 * rng.random(n), x + 0.01, x - 0.1, x + 0.1)
    df0 = rng.standard_normal(n)
    dg1 = np.full(n, 1.0 / n)
    for g1 in (0.01, -0.5):  # violated (lam > 0), inactive (lam = 0)
        xs, L, U, lam = O.mma_update(3, x, x - 0.02 * rng.random(n), x + 0.01, x - 0.1, x + 0.1, df0, g1, dg1)
        alpha, beta, p0, q0, p1, q1, r1 = O.mma_subproblem(x, L, U, df0, g1, dg1)
        P, Q = p0 + lam * p1, q0 + lam * q1
        d = P / (U - xs) ** 2 - Q / (xs - L) ** 2
        scale = P / (U - xs) ** 2 + Q / (xs - L) ** 2
        free = (xs > alpha + 1e-12) & (xs < beta - 1e-12)
        assert np.all(np.abs(d[free]) <= 1e-9 * scale[free])
        assert np.all(d[xs <= alpha + 1e-12] >= -1e-9 * scale[xs <= alpha + 1e-12])
        assert np.all(d[xs >= beta - 1e-12] <= 1e-9 * scale[xs >= beta - 1e-12])
        gval = np.sum(p1 / (U - xs) + q1 / (xs - L)) + r1
        if g1 > 0:
            assert lam > 0 and abs(gval) < 1e-10
        else:
            assert lam == 0 and gval <= 0


def test_mma_dual_maximum_by_scan():
    """The multiplier maximises the dual W(lam) = min_x [f0~ + lam g1~] over lam >= 0: a fine scan
    around it finds no larger value."""
    rng = np.random.default_rng(5)
    n = 500
    x = rng.uniform(0.2, 0.8, n)
    df0, dg1 = rng.standard_normal(n), np.full(n, 1.0 / n)
    xs, L, U, lam = O.mma_update(1, x, x, x, x, x, df0, 0.01, dg1)
    assert 0 < lam < 1e30
    alpha, beta, p0, q0, p1, q1, r1 = O.mma_subproblem(x, L, U, df0, 0.01, dg1)

    def W(lmb):
        xv = O.mma_x_of(lmb, L, U, alpha, beta, p0, q0, p1, q1)
        return np.sum((p0 + lmb * p1) / (U - xv) + (q0 + lmb * q1) / (xv - L)) + lmb * r1
    w0 = W(lam)
    for lmb in lam * np.linspace(0.9, 1.1, 201):
        assert W(lmb) <= w0 + 1e-12 * abs(w0)


def test_mma_infeasible_step_takes_the_most_feasible_point():
    """A violation the move limits cannot remove: the multiplier stops at its cap and the step goes
    to the minimiser of the approximated constraint alone in the subproblem's box (its lam -> inf
    limit: x = (sqrt(p1) L + sqrt(q1) U) / (sqrt(p1) + sqrt(q1)), clipped)."""
    rng = np.random.default_rng(7)
    n = 300
    x = rng.uniform(0.3, 0.7, n)
    df0, dg1 = rng.standard_normal(n), np.full(n, 1.0 / n)
    xs, L, U, lam = O.mma_update(1, x, x, x, x, x, df0, 0.5, dg1)
    alpha, beta, p0, q0, p1, q1, r1 = O.mma_subproblem(x, L, U, df0, 0.5, dg1)
    assert np.isfinite(lam) and lam >= 1e39
    limit = np.clip((np.sqrt(p1) * L + np.sqrt(q1) * U) / (np.sqrt(p1) + np.sqrt(q1)), alpha, beta)
    assert np.allclose(xs, limit, rtol=0, atol=1e-12)
    assert np.sum(p1 / (U - xs) + q1 / (xs - L)) + r1 > 0  # still violated: infeasible step


# ---------------------------------------------------------------- damped Jacobi smoother (variant)
def test_jacobi_damps_laplacian_modes_by_the_closed_form():
    """On the 1-D Dirichlet Laplacian (D = 2/h^2) each sine mode sin(k pi x) is an eigenvector
    of I - omega D^{-1} A with eigenvalue 1 - omega (1 - cos(k pi h)): nu sweeps from the mode
    (b = 0) multiply it by that factor to the nu-th power."""
    n = 31
    h = 1.0 / (n + 1)
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h ** 2
    xg = np.arange(1, n + 1) * h
    for k, omega, nu in ((1, 0.7, 3), (7, 0.5, 2), (30, 0.8, 4)):
        e = np.sin(k * np.pi * xg)
        out = O.jacobi_smooth(A, np.zeros(n), e, nu, omega)
        fac = (1.0 - omega * (1.0 - np.cos(k * np.pi * h))) ** nu
        np.testing.assert_allclose(out, fac * e, rtol=1e-12, atol=1e-14)


def test_jacobi_fixed_point_and_first_sweep():
    """The solution is a fixed point of the sweep; from zero the first sweep is omega D^{-1} b."""
    rng = np.random.default_rng(5)
    A = sp.random(40, 40, density=0.1, random_state=5) + sp.diags(5.0 + rng.random(40))
    b = rng.standard_normal(40)
    x = np.linalg.solve(A.toarray(), b)
    np.testing.assert_allclose(O.jacobi_smooth(A, b, x, 3, 0.7), x, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(O.jacobi_smooth(A, b, np.zeros(40), 1, 0.6), 0.6 * b / A.diagonal(), rtol=1e-15)


def test_jacobi_vcycle_contracts_and_single_level_is_two_smoothings():
    """With damped Jacobi smoothing the V-cycle of a space-time problem contracts (rate below 0.7
    over eight cycles); on a two-level hierarchy it equals the hand composition."""
    mat = O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
    m = O.Mesh((16, 16), 16, mat=mat, bc="patch_left", bc_width=0.2)
    g = np.random.default_rng(2).random((16, 16))
    mg = O.build_mg(m, g, O.hierarchy(m, coarse_cap=300))
    A = mg[0].A
    f = O.assemble_source(m, O.source_fn("uniform", 1.0))
    x = np.zeros_like(f)
    res = [np.linalg.norm(f)]
    for _ in range(8):
        x = x + O.vcycle(mg, f - A @ x, nsmooth=2, smoother="jacobi", omega=0.7)
        res.append(np.linalg.norm(f - A @ x))
    assert (res[-1] / res[0]) ** (1 / 8) < 0.7, res
    two = O.build_mg(m, g, O.hierarchy(m, n_levels=2))
    b = np.random.default_rng(3).standard_normal(m.n_nodes)
    b[two[0].mask] = 0
    A0, Pt = two[0].A, two[0].Pt
    x1 = O.jacobi_smooth(A0, b, np.zeros_like(b), 2, 0.7)
    xc = np.linalg.solve(two[1].A.toarray(), Pt.T @ (b - A0 @ x1))
    x2 = O.jacobi_smooth(A0, b, x1 + Pt @ xc, 2, 0.7)
    np.testing.assert_allclose(O.vcycle(two, b, nsmooth=2, smoother="jacobi", omega=0.7), x2, rtol=1e-13, atol=1e-15)


def test_jacobi_damping_half_keeps_a_space_time_vcycle_convergent():
    """The reading of the default damping: on a space-time design (paper material, 40 x 24 x 20)
    the stationary Jacobi-smoothed V-cycle (nu = 2) contracts with omega = 0.5 and diverges with
    omega = 0.7."""
    m = O.Mesh((40, 24), 20, mat=O.Material(), bc="patch_left", bc_width=0.3)
    g = np.random.default_rng(100).random(m.elem_shape)
    mg = O.build_mg(m, g, O.hierarchy(m, coarse_cap=300))
    A = mg[0].A
    f = O.assemble_source(m, O.source_fn("uniform", 1.0))
    ratio = {}
    for w in (0.5, 0.7):
        x = np.zeros_like(f)
        for _ in range(8):
            x = x + O.vcycle(mg, f - A @ x, nsmooth=2, smoother="jacobi", omega=w)
        ratio[w] = np.linalg.norm(f - A @ x) / np.linalg.norm(f)
    assert ratio[0.5] < 0.05 and ratio[0.7] > 100.0, ratio
