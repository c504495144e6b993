"""GPU parity: every kernel family through the C ABI against the FP64 CPU oracle.

Sizes are chosen so the oracle finishes in seconds while the meshes span several
32x8 thread tiles with ragged edges (node counts not multiples of the tile), both
spatial dimensions (2+1D and 3+1D), both design layouts and every boundary kind.

Tolerances.  FP64 operators, transfers and diagonals: relative 1e-12 to 1e-14 of the largest
entry and, row by row, the componentwise rounding bound c u |J|_elem |x| (u = 2^-53).  FP32
operators and transfers: row by row within c u |J|_elem |x| with u = 2^-24, |J|_elem the
element-wise absolute operator (its Galerkin products on coarse levels) and c the number of
summed terms plus a margin, so an error in a small (insulating) term of any row shows.  The
FP32 operator is compared with the oracle operator of the design it reads (FP64 design for
the FP32 27-point stencils of time-constant 2-D designs, BF16-rounded design otherwise).
FP32 smoothing and V-cycles: the GPU result's error against the FP64 oracle must stay within
a small multiple of the error of the oracle's own float32 run of the same algorithm (and
below 5e-3).  Solves: 1e-10 at rtol = max(1e-13, 20x the FP64 residual floor of the case).
"""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import (U32, U64, bf16_round, ensure_built, galerkin_abs, gpu_mesh, parity_rtol,
                               rel_err, rowwise_excess)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATS = {
    "paper": O.Material(),
    "unitcap": O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3),
    "capvar": O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3),
}

# (ns, nt, material, bc, bc_width, space-time design?)
CASES = [
    ((40, 24), 20, "paper", "patch_left", 0.3, True),
    ((36, 20), 16, "unitcap", "patch_bottom", 0.25, False),
    ((16, 16), 24, "paper", "all_walls", 0.1, False),
    ((6, 4, 8), 6, "capvar", "patch_left", 0.5, False),
    ((4, 6, 4), 5, "paper", "none", 0.1, True),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


def _case(i, seed=0):
    ns, nt, mat, bc, w, st = CASES[i]
    om = O.Mesh(ns, nt, mat=MATS[mat], bc=bc, bc_width=w)
    rng = np.random.default_rng(100 + i + seed)
    g = rng.random(om.elem_shape if st else tuple(reversed(ns)))
    return om, g


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _fp32_design(om, g):
    """Design the FP32 level-0 operator is built from: extruded 2-D designs are applied as
    FP32 27-point stencils computed from the FP64 design; all other cases read the BF16 design."""
    extruded = g.size == int(np.prod(om.ns))
    return g if (extruded and om.sd == 2) else bf16_round(g)


@pytest.mark.parametrize("i", range(len(CASES)))
@pytest.mark.parametrize("transpose", [False, True])
def test_fine_operator_fp64_and_fp32(i, transpose):
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=400)
    gm.set_design(g)
    A = O.assemble(om, g)
    A = A.T.tocsr() if transpose else A
    x = np.random.default_rng(1).standard_normal(om.n_nodes)
    y = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
    gm.apply(0, _dev(x), y, "fp64", transpose)
    assert rel_err(y.cpu().numpy(), A @ x) < 1e-13
    B = O.abs_operator(om, g)
    B = B.T.tocsr() if transpose else B
    assert rowwise_excess(y.cpu().numpy(), A @ x, B, x, 80, U64) <= 1.0
    # FP32 operator (BF16 design, or FP32 stencils for extruded 2-D designs), row by row
    g32 = _fp32_design(om, g)
    A16 = O.assemble(om, g32)
    A16 = A16.T.tocsr() if transpose else A16
    B16 = O.abs_operator(om, g32)
    B16 = B16.T.tocsr() if transpose else B16
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
    gm.apply(0, _dev(x, torch.float32), y32, "mixed", transpose)
    c = 80 if om.sd == 2 else 280  # summed terms per row (64 or 256) plus a margin
    assert rowwise_excess(y32.cpu().numpy(), A16 @ x32, B16, x32, c, U32) <= 1.0
    d = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
    gm.diag(0, d, "fp64")
    assert rel_err(d.cpu().numpy(), A.diagonal()) < 1e-14


@pytest.mark.parametrize("i", range(len(CASES)))
def test_hierarchy_galerkin_transfers(i):
    """Every level: the coarse operator apply (both orientations), its diagonal, and the
    masked restriction / prolongation against P^T A P + (I - D_c) built by sparse products."""
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    glev = gm.levels()
    olev = O.hierarchy(om, coarse_cap=300)
    assert [(tuple(L.ns), L.nt, L.to_next) for L in olev] == [(L["ns"], L["nt"], L["to_next"]) for L in glev]
    mg = O.build_mg(om, g, olev)
    rng = np.random.default_rng(2)
    B = O.abs_operator(om, g)  # element-wise absolute operator, then its Galerkin products
    c_op = 80 if om.sd == 2 else 280
    for l in range(len(mg)):
        N = mg[l].A.shape[0]
        x = rng.standard_normal(N)
        x32 = x.astype(np.float32).astype(np.float64)
        if l > 0:
            B = galerkin_abs(B, mg[l - 1].Pt, mg[l].mask)
        for tr in (False, True):
            A = mg[l].A.T.tocsr() if tr else mg[l].A
            Bt = B.T.tocsr() if tr else B
            y = torch.empty(N, dtype=torch.float64, device="cuda")
            gm.apply(l, _dev(x), y, "fp64", tr)
            assert rel_err(y.cpu().numpy(), A @ x) < 1e-12, (l, tr)
            if l > 0:
                y32 = torch.empty(N, dtype=torch.float32, device="cuda")
                gm.apply(l, _dev(x, torch.float32), y32, "mixed", tr)
                assert rowwise_excess(y32.cpu().numpy(), A @ x32, Bt, x32, c_op, U32) <= 1.0, (l, tr)
        d = torch.empty(N, dtype=torch.float64, device="cuda")
        gm.diag(l, d, "fp64")
        assert rel_err(d.cpu().numpy(), mg[l].A.diagonal()) < 1e-12
        if l + 1 < len(mg):
            Pt = mg[l].Pt
            rc = torch.empty(Pt.shape[1], dtype=torch.float64, device="cuda")
            gm.restrict(l, _dev(x), rc, "fp64")
            assert rel_err(rc.cpu().numpy(), Pt.T @ x) < 1e-14
            assert rowwise_excess(rc.cpu().numpy(), Pt.T @ x, Pt.T, x, 32, U64) <= 1.0
            rc32 = torch.empty(Pt.shape[1], dtype=torch.float32, device="cuda")
            gm.restrict(l, _dev(x, torch.float32), rc32, "mixed")
            assert rowwise_excess(rc32.cpu().numpy(), Pt.T @ x32, Pt.T, x32, 32, U32) <= 1.0, l
            xc = rng.standard_normal(Pt.shape[1])
            xf0 = rng.standard_normal(N)
            xf = _dev(xf0)
            gm.prolong(l, _dev(xc), xf, "fp64")
            assert rel_err(xf.cpu().numpy(), xf0 + Pt @ xc) < 1e-14
            # FP32 prolongation x_f += P x_c: within 32 u32 (|x_f| + P |x_c|) per row
            xc32 = xc.astype(np.float32).astype(np.float64)
            xf032 = xf0.astype(np.float32).astype(np.float64)
            xf32 = _dev(xf0, torch.float32)
            gm.prolong(l, _dev(xc, torch.float32), xf32, "mixed")
            bound = 32 * U32 * (np.abs(xf032) + Pt @ np.abs(xc32)) + 1e-300
            assert (np.abs(xf32.cpu().numpy() - (xf032 + Pt @ xc32)) <= bound).all(), l
    Ainv = gm.coarse_inverse()
    Ac = mg[-1].A.toarray()
    assert np.abs(Ainv @ Ac - np.eye(Ac.shape[0])).max() < 1e-9


@pytest.mark.parametrize("i", [0, 1, 3])
@pytest.mark.parametrize("zero_init", [True, False])
def test_smoother_matches_oracle_gmres(i, zero_init):
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    olev = O.hierarchy(om, coarse_cap=300)
    mg = O.build_mg(om, g, olev)
    rng = np.random.default_rng(3)
    for l in (0, 1):
        A = mg[l].A
        b = rng.standard_normal(A.shape[0])
        b[mg[l].mask] = 0
        x0 = np.zeros_like(b) if zero_init else 0.1 * rng.standard_normal(A.shape[0]) * (~mg[l].mask)
        for tr in (False, True):
            At = A.T.tocsr() if tr else A
            ref = O.gmres_jacobi(At, b, x0, 10)
            x = _dev(x0)
            gm.smooth(l, _dev(b), x, 10, zero_init, "fp64", tr)
            assert rel_err(x.cpu().numpy(), ref) < 1e-9, (l, tr)
            # FP32: the error against the FP64 oracle stays within a small multiple of the
            # error of the oracle's own float32 run of the same smoother on the same inputs
            x32 = _dev(x0, torch.float32)
            gm.smooth(l, _dev(b, torch.float32), x32, 10, zero_init, "mixed", tr)
            A32 = O.assemble(om, _fp32_design(om, g)) if l == 0 else A
            A32 = A32.T.tocsr() if tr else A32
            b32 = b.astype(np.float32).astype(np.float64)
            x032 = x0.astype(np.float32).astype(np.float64)
            ref32 = O.gmres_jacobi(A32, b32, x032, 10)
            emu = O.gmres_jacobi(A32, b32, x032, 10, dtype=np.float32)
            e_gpu, e_emu = rel_err(x32.cpu().numpy(), ref32), rel_err(emu, ref32)
            assert e_gpu <= max(FP32_FACTOR * e_emu, 64 * U32) and e_gpu < 5e-3, (l, tr, e_gpu, e_emu)


def test_smoother_zero_rhs_leaves_zero():
    om, g = _case(1)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    b = torch.zeros(om.n_nodes, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    gm.smooth(0, b, x, 10, True, "fp64")
    assert torch.count_nonzero(x).item() == 0


# A single-precision run on the GPU may differ from the oracle's float32 run in summation
# order (blocked reductions, classical instead of modified Gram-Schmidt), so its error against
# the FP64 oracle is bounded by this multiple of the oracle float32 run's error.
FP32_FACTOR = 10.0


def _mixed_levels(om, g, mg):
    """The operators of the mixed V-cycle: level 0 from the design the FP32 level-0 kernels
    read, coarse levels the FP64 Galerkin operators (rounded to FP32 by the float32 run)."""
    A0 = O.assemble(om, _fp32_design(om, g))
    return [O.MGLevel(mg[0].level, A0, mg[0].mask, mg[0].Pt)] + list(mg[1:])


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_mixed_vcycle_matches_float32_oracle(i):
    """The mixed-precision V-cycle (FP32 smoothing, residuals and transfers, FP64 coarsest
    solve) against the oracle's V-cycle on the same operators: its error stays within a small
    multiple of the oracle's own float32 V-cycle error, both orientations."""
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    mg = _mixed_levels(om, g, O.build_mg(om, g, O.hierarchy(om, coarse_cap=300)))
    b = np.random.default_rng(4).standard_normal(om.n_nodes)
    b[mg[0].mask] = 0
    b32 = b.astype(np.float32).astype(np.float64)
    for tr in (False, True):
        ref = O.vcycle(mg, b32, transpose=tr)
        emu = O.vcycle(mg, b32, transpose=tr, dtype=np.float32)
        x = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.vcycle(_dev(b, torch.float32), x, "mixed", tr)
        e_gpu, e_emu = rel_err(x.cpu().numpy(), ref), rel_err(emu, ref)
        assert e_gpu <= max(FP32_FACTOR * e_emu, 64 * U32) and e_gpu < 5e-3, (tr, e_gpu, e_emu)


@pytest.mark.parametrize("i", [0, 1, 3])
def test_vcycle_matches_oracle(i):
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    mg = O.build_mg(om, g, O.hierarchy(om, coarse_cap=300))
    b = np.random.default_rng(4).standard_normal(om.n_nodes)
    b[mg[0].mask] = 0
    for tr in (False, True):
        ref = O.vcycle(mg, b, transpose=tr)
        x = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.vcycle(_dev(b), x, "fp64", tr)
        assert rel_err(x.cpu().numpy(), ref) < 1e-8, tr


def _src_kw(kind):
    return dict(kind=kind, q0=1.0, a=1.0, b=0.5, f=4.0)


@pytest.mark.parametrize("i", range(len(CASES)))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forward_adjoint_sensitivities(i, precision):
    om, g = _case(i)
    src = "sin_t" if i % 2 == 0 else "uniform"
    sol = O.forward(om, g, src, 1.0)
    dm = O.dirichlet_mask(om)
    lam = O.adjoint(sol.A, sol.f, dm, sol.lu)
    sens = O.sensitivities(om, g, sol.s, lam, extruded=g.size == int(np.prod(om.ns)))
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    rt = parity_rtol(sol.A, sol.s, sol.f)
    st = gm.solve_forward(rtol=rt, precision=precision, max_it=400, **_src_kw(src))
    assert st["converged"] and st["rel_res"] <= rt
    np.testing.assert_allclose(gm.state("rhs"), sol.f, rtol=0, atol=1e-14 * np.abs(sol.f).max())
    s = gm.state("T")
    assert rel_err(s, sol.s) < 1e-10
    phi, sta = gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision=precision,
                                max_it=400)
    assert sta["converged"]
    np.testing.assert_allclose(phi, O.compliance(sol.f, sol.s), rtol=1e-11)
    assert rel_err(gm.state("lambda"), lam) < 1e-10
    gs = gm.sensitivities()
    assert rel_err(gs, sens.reshape(-1)) < 1e-9


def test_pnorm_objective_and_adjoint():
    om, g = _case(0)
    sol = O.forward(om, g, "uniform", 1.0)
    dm = O.dirichlet_mask(om)
    phi_ref, dphi = O.pnorm(om, sol.s, 20)
    lam = O.adjoint(sol.A, dphi, dm, sol.lu)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision="fp64", max_it=400)
    phi, st = gm.solve_adjoint("pnorm", P=20, rtol=parity_rtol(sol.A.T, lam, dphi), precision="fp64", max_it=400)
    np.testing.assert_allclose(phi, phi_ref, rtol=1e-11)
    np.testing.assert_allclose(gm.state("adj_rhs"), np.where(dm, 0, dphi), rtol=1e-11, atol=1e-14 * np.abs(dphi).max())
    assert rel_err(gm.state("lambda"), lam) < 1e-10


def test_mixed_to_1e8_meets_1e6_and_fp64_meets_1e10():
    """Target tolerances at the 1e-8 outer residual: the mixed path's temperature error
    against the FP64 oracle is reported and must be below 1e-6 (relative, max norm)."""
    om, g = _case(1)
    sol = O.forward(om, g, "uniform", 1.0)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    st = gm.solve_forward(rtol=1e-8, precision="mixed")
    assert st["converged"] and st["rel_res"] <= 1e-8
    assert rel_err(gm.state("T"), sol.s) < 1e-6
    # the FP32 preconditioner costs no outer iterations: at most one more than all-FP64
    st64 = gm.solve_forward(rtol=1e-8, precision="fp64")
    assert st64["converged"] and st["outer_its"] <= st64["outer_its"] + 1, (st["outer_its"], st64["outer_its"])
    st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision="fp64", max_it=400)
    assert rel_err(gm.state("T"), sol.s) < 1e-10


def test_c0_workload_compliance():
    """32x32x32 (33^3 DOFs), uniform design 0.5, unit capacity, FP64: compliance and state."""
    import workloads as W
    w = W.C0
    om = O.Mesh(w.ns, w.nt, mat=O.Material(**w.material), bc=w.bc, bc_width=w.bc_width)
    g = W.make_design(w)
    sol = O.forward(om, g, "uniform", w.source_q0)
    gm = gpu_mesh(om)
    gm.set_design(g)
    assert [L["ns"] + (L["nt"],) for L in gm.levels()] == [(32, 32, 32), (16, 16, 32), (16, 16, 16), (8, 8, 16)]
    st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision="fp64", max_it=400)
    assert rel_err(gm.state("T"), sol.s) < 1e-10
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    phi, _ = gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision="fp64", max_it=400)
    np.testing.assert_allclose(phi, O.compliance(sol.f, sol.s), rtol=1e-11)
    assert rel_err(gm.state("lambda"), lam) < 1e-10


def test_warm_start_and_errors():
    from paper_2508_09589_gb300 import STError
    om, g = _case(1)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    with pytest.raises(STError):
        gm.solve_forward()  # no design yet
    gm.set_design(g)
    with pytest.raises(STError):
        gm.set_design(np.zeros(7))  # wrong size
    st1 = gm.solve_forward(rtol=1e-10)
    st2 = gm.solve_forward(rtol=1e-10, warm_start=True)
    assert st2["outer_its"] <= 1
    st3 = gm.solve_forward(rtol=1e-14, max_it=1, allow_not_converged=True)
    assert st3["status"] == -3 and not st3["converged"]
    assert st1["converged"]


def test_graphs_and_eager_identical():
    om, g = _case(0)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    gm.solve_forward(rtol=1e-9, use_graphs=False)
    a = gm.state("T")
    gm.solve_forward(rtol=1e-9, use_graphs=True)
    b = gm.state("T")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("i", [0, 3])
def test_apply_timer_counts_level0_applies_and_changes_nothing(i):
    """The event timer records every level-0 smoother apply (2 sweeps x 10 steps per outer
    iteration, graphs and eager) and leaves the solution bit for bit unchanged."""
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    for graphs in (True, False):
        gm.solve_forward(rtol=1e-9, use_graphs=graphs)
        a = gm.state("T")
        gm.apply_timer(True)
        st = gm.solve_forward(rtol=1e-9, use_graphs=graphs)
        ms, n = gm.apply_timer_read()
        gm.apply_timer(False)
        np.testing.assert_array_equal(gm.state("T"), a)
        assert n == 2 * 10 * st["outer_its"]
        assert ms > 0
        phi, sa = gm.solve_adjoint()
        assert gm.apply_timer_read() == (ms, n)  # stopped: totals kept, nothing added


@pytest.mark.parametrize("i", [0, 1, 3])
def test_persistent_tail_matches_launch_per_phase(i, monkeypatch):
    """The V-cycle run as one persistent cooperative kernel (small levels) and as one launch
    per phase give the same preconditioner output (FP64: rounding-level differences only)."""
    om, g = _case(i)
    b = np.random.default_rng(9).standard_normal(om.n_nodes)
    b[O.dirichlet_mask(om)] = 0
    out = []
    for nodes in ("0", "100000000"):
        monkeypatch.setenv("ST_VTAIL_NODES", nodes)
        gm = gpu_mesh(om, coarse_dof_cap=300)
        gm.set_design(g)
        x = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.vcycle(_dev(b), x, "fp64", False)
        out.append(x.cpu().numpy())
        st = gm.solve_forward(rtol=1e-10, precision="mixed")
        assert st["converged"]
    assert rel_err(out[1], out[0]) < 1e-11


@pytest.mark.parametrize("i", [1, 2])
@pytest.mark.parametrize("blocks", [1, 12, 18, 30])
def test_march_kernels_with_long_and_ragged_time_chunks(i, blocks):
    """The time-marching stencil kernels with thread-block budgets that give each block the
    whole time axis or chunks of 9, 6 or 4 planes with a ragged last chunk: operator,
    smoother and full forward / adjoint solves against the oracle."""
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300, march_blocks=blocks)
    gm.set_design(g)
    A = O.assemble(om, g)
    x = np.random.default_rng(11).standard_normal(om.n_nodes)
    for tr in (False, True):
        At = A.T.tocsr() if tr else A
        y = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.apply(0, _dev(x), y, "fp64", tr)
        assert rel_err(y.cpu().numpy(), At @ x) < 1e-13
        y32 = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.apply(0, _dev(x, torch.float32), y32, "mixed", tr)
        x32 = x.astype(np.float32).astype(np.float64)
        B = O.abs_operator(om, g)
        assert rowwise_excess(y32.cpu().numpy(), At @ x32, B.T.tocsr() if tr else B, x32, 80, U32) <= 1.0
        b = x * (~O.dirichlet_mask(om))
        ref = O.gmres_jacobi(At, b, np.zeros_like(b), 10)
        xs = torch.zeros(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.smooth(0, _dev(b), xs, 10, True, "fp64", tr)
        assert rel_err(xs.cpu().numpy(), ref) < 1e-9
    sol = O.forward(om, g, "uniform", 1.0)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    for precision in ("fp64", "mixed"):
        st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision=precision, max_it=400)
        assert st["converged"]
        assert rel_err(gm.state("T"), sol.s) < (1e-10 if precision == "fp64" else 1e-6)
        gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision=precision, max_it=400)
        assert rel_err(gm.state("lambda"), lam) < (1e-10 if precision == "fp64" else 1e-6)


def test_coarse_gmres_single_level_reaches_its_tolerance():
    """One-level hierarchy: the V-cycle is the coarsest Jacobi-GMRES solve alone; its output
    meets the requested relative residual (and converges to the exact solve when tight)."""
    om = O.Mesh((10, 6), 4, mat=MATS["unitcap"], bc="patch_bottom", bc_width=0.3)
    g = np.random.default_rng(12).random((6, 10))
    A = O.assemble(om, g)
    b = np.random.default_rng(12).standard_normal(om.n_nodes)
    b[O.dirichlet_mask(om)] = 0
    exact = O.solve_direct(A, b)
    for rtol, it in ((1e-6, 400), (1e-12, 2000)):
        gm = gpu_mesh(om, max_levels=1, coarse_solver="gmres", coarse_rtol=rtol, coarse_max_it=it)
        gm.set_design(g)
        assert len(gm.levels()) == 1
        x = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.vcycle(_dev(b), x, "fp64", False)
        xh = x.cpu().numpy()
        assert np.linalg.norm(b - A @ xh) <= 1.5 * rtol * np.linalg.norm(b)
        if rtol < 1e-9:
            assert rel_err(xh, exact) < 1e-8
        with pytest.raises(Exception):
            gm.coarse_inverse()


@pytest.mark.parametrize("i", [0, 1, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coarse_gmres_solver_forward_adjoint(i, precision):
    """The paper's coarsest solve (Jacobi-GMRES to 1e-6) inside the V-cycle: FGMRES reaches
    the same solution and adjoint as with the dense coarsest inverse."""
    om, g = _case(i)
    sol = O.forward(om, g, "uniform", 1.0)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    gm = gpu_mesh(om, coarse_dof_cap=300, coarse_solver="gmres")
    gm.set_design(g)
    st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision=precision, max_it=400)
    assert st["converged"]
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert rel_err(gm.state("T"), sol.s) < tol
    gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision=precision, max_it=400)
    assert rel_err(gm.state("lambda"), lam) < tol


def test_coarse_solver_switches_to_gmres_above_the_dense_cap():
    """Odd element counts stop Algorithm 1 at once: the 46 x 46 x 18-node level cannot use
    the dense inverse (more than 4096 nodes), so the default picks Jacobi-GMRES."""
    om = O.Mesh((45, 45), 17, mat=MATS["unitcap"], bc="patch_left", bc_width=0.1)
    g = np.random.default_rng(13).random((45, 45))
    sol = O.forward(om, g, "uniform", 1.0)
    gm = gpu_mesh(om)
    assert len(gm.levels()) == 1 and om.n_nodes > 4096
    gm.set_design(g)
    for precision in ("fp64", "mixed"):
        st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision=precision, max_it=400)
        assert st["converged"]
        assert rel_err(gm.state("T"), sol.s) < (1e-10 if precision == "fp64" else 1e-6)
    with pytest.raises(Exception):
        gpu_mesh(om, coarse_solver="dense")


@pytest.mark.parametrize("nt", [1, 2, 3, 4, 5, 6])
def test_few_time_planes_smoother_and_solve(nt):
    """Time-constant 2-D designs with 1..6 time elements: every plane of the smoothing level
    is a first, second, last or second-to-last plane, so the stencil smoother runs on its
    boundary-plane path only (and n_t = 1 uses the single-slab class); the fine level has more
    than 15,000 nodes, so FP32 smoothing uses the scaled stencil kernel as well."""
    om = O.Mesh((180, 48), nt, mat=MATS["unitcap"], bc="patch_left", bc_width=0.2)
    g = np.random.default_rng(30 + nt).random((48, 180))
    gm = gpu_mesh(om, coarse_dof_cap=600)
    gm.set_design(g)
    levels = gm.levels()
    assert len(levels) >= 2
    A = O.assemble(om, g)
    b = np.random.default_rng(31).standard_normal(om.n_nodes)
    b[O.dirichlet_mask(om)] = 0
    for tr in (False, True):
        At = A.T.tocsr() if tr else A
        ref = O.gmres_jacobi(At, b, np.zeros_like(b), 10)
        x = torch.zeros(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.smooth(0, _dev(b), x, 10, True, "fp64", tr)
        assert rel_err(x.cpu().numpy(), ref) < 1e-9
        x32 = torch.zeros(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.smooth(0, _dev(b, torch.float32), x32, 10, True, "mixed", tr)
        b32 = b.astype(np.float32).astype(np.float64)
        ref32 = O.gmres_jacobi(At, b32, np.zeros_like(b), 10)
        emu = O.gmres_jacobi(At, b32, np.zeros_like(b), 10, dtype=np.float32)
        e_gpu, e_emu = rel_err(x32.cpu().numpy(), ref32), rel_err(emu, ref32)
        assert e_gpu <= max(FP32_FACTOR * e_emu, 64 * U32) and e_gpu < 5e-3, (tr, e_gpu, e_emu)
    sol = O.forward(om, g, "uniform", 1.0)
    for precision in ("fp64", "mixed"):
        st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision=precision, max_it=400)
        assert st["converged"]
        assert rel_err(gm.state("T"), sol.s) < 1e-10


@pytest.mark.parametrize("i", [0, 1, 3])
def test_full_coarsening_hierarchy_and_solves(i):
    """Full space-time coarsening (both directions halved on every level, the ablation of Sec.
    5.1.2): the hierarchy, every level's Galerkin operator and transfers, and the forward and
    adjoint solves match the oracle in FP64 and mixed precision."""
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300, coarsening="full")
    gm.set_design(g)
    olev = O.hierarchy(om, coarse_cap=300, mode="full")
    assert [(tuple(L.ns), L.nt, L.to_next) for L in olev] == [(L["ns"], L["nt"], L["to_next"]) for L in gm.levels()]
    mg = O.build_mg(om, g, olev)
    rng = np.random.default_rng(5)
    for l in range(len(mg)):
        N = mg[l].A.shape[0]
        x = rng.standard_normal(N)
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        gm.apply(l, _dev(x), y, "fp64")
        assert rel_err(y.cpu().numpy(), mg[l].A @ x) < 1e-12, l
        if l + 1 < len(mg):
            Pt = mg[l].Pt
            rc = torch.empty(Pt.shape[1], dtype=torch.float64, device="cuda")
            gm.restrict(l, _dev(x), rc, "fp64")
            assert rel_err(rc.cpu().numpy(), Pt.T @ x) < 1e-14
    sol = O.forward(om, g, "uniform", 1.0)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    for precision in ("fp64", "mixed"):
        st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision=precision, max_it=600)
        assert st["converged"]
        assert rel_err(gm.state("T"), sol.s) < (1e-10 if precision == "fp64" else 1e-6)
        gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision=precision, max_it=600)
        assert rel_err(gm.state("lambda"), lam) < (1e-10 if precision == "fp64" else 1e-6)
