"""The time-marching element kernels of space-time 2-D designs in FP32: level 0 (k_l0st.cu) and the
levels reached by coarsening space only (k_lcst.cu): operator apply, smoother apply and start,
residual inside the mixed V-cycle, and mixed solves, against the oracle; and the FP64 outer
operator on its marching kernel (k_fg_march.cu). Cases: ragged 32 x 8 tiles in both axes, every
boundary kind, one to few time slabs, and thread-block budgets that give each block the whole
time axis or short time chunks with a ragged last chunk."""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import (U32, U64, bf16_round, ensure_built, galerkin_abs, gpu_mesh, parity_rtol, rel_err,
                               rowwise_excess)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)

# (ns, nt, bc, bc_width, march_blocks)
CASES = [
    ((40, 24), 20, "patch_left", 0.3, 0),
    ((72, 34), 8, "patch_bottom", 0.25, 0),
    ((70, 33), 9, "patch_left", 0.4, 30),
    ((16, 16), 3, "all_walls", 0.1, 0),
    ((33, 9), 1, "none", 0.1, 0),
    ((40, 24), 20, "patch_left", 0.3, 6),
    ((96, 40), 12, "all_walls", 0.1, 1),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _case(i):
    ns, nt, bc, w, blocks = CASES[i]
    om = O.Mesh(ns, nt, mat=MAT, bc=bc, bc_width=w)
    g = np.random.default_rng(700 + i).random(om.elem_shape)
    gm = gpu_mesh(om, coarse_dof_cap=300, march_blocks=blocks)
    gm.set_design(g, "spacetime")  # explicit: with one slab the counts of both layouts agree
    return om, g, gm


@pytest.mark.parametrize("i", range(len(CASES)))
def test_fp32_apply_rowwise(i):
    """y = A x and A^T x in FP32 within c u32 (|J|_elem |x|)_i of the oracle on the BF16 design,
    row by row (prescribed rows: the identity, exact)."""
    om, g, gm = _case(i)
    g16 = bf16_round(g)
    A = O.assemble(om, g16)
    B = O.abs_operator(om, g16)
    x = np.random.default_rng(5 + i).standard_normal(om.n_nodes)
    x32 = x.astype(np.float32).astype(np.float64)
    for tr in (False, True):
        At = A.T.tocsr() if tr else A
        y = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.apply(0, _dev(x, torch.float32), y, "mixed", tr)
        yv = y.cpu().numpy().astype(np.float64)
        assert rowwise_excess(yv, At @ x32, B.T.tocsr() if tr else B, x32, 80, U32) <= 1.0, tr
        mask = O.dirichlet_mask(om)
        assert np.array_equal(yv[mask], x32[mask])


@pytest.mark.parametrize("i", range(len(CASES)))
@pytest.mark.parametrize("zero_init", [True, False])
def test_fp32_smoother(i, zero_init):
    """Jacobi-GMRES(10) at level 0 in FP32 (apply w = A D^-1 u; from a nonzero iterate also the
    start u_0 = b - A x): its error against the FP64 oracle stays within 10x the error of the
    oracle's own float32 run on the same inputs."""
    om, g, gm = _case(i)
    A = O.assemble(om, bf16_round(g))
    mask = O.dirichlet_mask(om)
    rng = np.random.default_rng(9 + i)
    b = rng.standard_normal(om.n_nodes)
    b[mask] = 0
    x0 = np.zeros_like(b) if zero_init else 0.1 * rng.standard_normal(om.n_nodes) * (~mask)
    b32 = b.astype(np.float32).astype(np.float64)
    x032 = x0.astype(np.float32).astype(np.float64)
    for tr in (False, True):
        At = A.T.tocsr() if tr else A
        ref = O.gmres_jacobi(At, b32, x032, 10)
        emu = O.gmres_jacobi(At, b32, x032, 10, dtype=np.float32)
        x = _dev(x0, torch.float32)
        gm.smooth(0, _dev(b, torch.float32), x, 10, zero_init, "mixed", tr)
        e_gpu, e_emu = rel_err(x.cpu().numpy(), ref), rel_err(emu, ref)
        assert e_gpu <= max(10.0 * e_emu, 64 * U32) and e_gpu < 5e-3, (tr, e_gpu, e_emu)


@pytest.mark.parametrize("i", [0, 1, 3, 6])
def test_mixed_vcycle_and_solves(i):
    """The mixed V-cycle (its level-0 residual and post-smoothing start are the marching
    kernels) against the oracle's float32 V-cycle, and mixed forward / adjoint solves to the
    oracle's direct solution."""
    om, g, gm = _case(i)
    lev = O.hierarchy(om, coarse_cap=300)
    mg = O.build_mg(om, g, lev)
    A0 = O.assemble(om, bf16_round(g))
    mgx = [O.MGLevel(mg[0].level, A0, mg[0].mask, mg[0].Pt)] + list(mg[1:])
    b = np.random.default_rng(4).standard_normal(om.n_nodes)
    b[mg[0].mask] = 0
    b32 = b.astype(np.float32).astype(np.float64)
    for tr in (False, True):
        ref = O.vcycle(mgx, b32, transpose=tr)
        emu = O.vcycle(mgx, b32, transpose=tr, dtype=np.float32)
        x = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.vcycle(_dev(b, torch.float32), x, "mixed", tr)
        e_gpu, e_emu = rel_err(x.cpu().numpy(), ref), rel_err(emu, ref)
        assert e_gpu <= max(10.0 * e_emu, 64 * U32) and e_gpu < 5e-3, (tr, e_gpu, e_emu)
    sol = O.forward(om, g, "uniform", 1.0)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    st = gm.solve_forward(rtol=1e-10, precision="mixed", max_it=400)
    assert st["converged"]
    assert rel_err(gm.state("T"), sol.s) < 1e-6
    gm.solve_adjoint("compliance", rtol=1e-10, precision="mixed", max_it=400)
    assert rel_err(gm.state("lambda"), lam) < 1e-6
    st64 = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision="fp64", max_it=400)
    assert st64["converged"] and rel_err(gm.state("T"), sol.s) < 1e-10


@pytest.mark.parametrize("i", [0, 1, 6])
def test_fp32_coarse_apply_rowwise(i):
    """Every level reached from level 0 by coarsening space only: y = A_l x and A_l^T x in FP32
    from the (slab, element) M and K rows extracted from the FP64 Galerkin blocks, within
    80 u32 (B_l |x|)_i of the oracle's P^T A P row by row (B_l the Galerkin products of
    |J|_elem), prescribed rows exact."""
    om, g, gm = _case(i)
    olev = O.hierarchy(om, coarse_cap=300)
    assert [(tuple(L.ns), L.nt, L.to_next) for L in olev] == [(L["ns"], L["nt"], L["to_next"])
                                                             for L in gm.levels()]
    mg = O.build_mg(om, g, olev)
    B = O.abs_operator(om, g)
    rng = np.random.default_rng(31 + i)
    checked = 0
    for l in range(1, len(mg)):
        if olev[l - 1].to_next != "space":
            break
        B = galerkin_abs(B, mg[l - 1].Pt, mg[l].mask)
        N = mg[l].A.shape[0]
        x = rng.standard_normal(N)
        x32 = x.astype(np.float32).astype(np.float64)
        for tr in (False, True):
            A = mg[l].A.T.tocsr() if tr else mg[l].A
            y = torch.empty(N, dtype=torch.float32, device="cuda")
            gm.apply(l, _dev(x, torch.float32), y, "mixed", tr)
            yv = y.cpu().numpy().astype(np.float64)
            assert rowwise_excess(yv, A @ x32, B.T.tocsr() if tr else B, x32, 80, U32) <= 1.0, (l, tr)
            assert np.array_equal(yv[mg[l].mask], x32[mg[l].mask])
        checked += 1
    assert checked >= 1


@pytest.mark.parametrize("i", range(len(CASES)))
def test_fp64_apply_rowwise(i):
    """The FP64 outer operator on the marching kernels (k_fg_march.cu, space-time 2-D): y = J x and
    J^T x from the FP64 design within 80 u64 (|J|_elem |x|)_i of the oracle row by row and 1e-13
    of the largest entry, prescribed rows exact."""
    om, g, gm = _case(i)
    A = O.assemble(om, g)
    B = O.abs_operator(om, g)
    x = np.random.default_rng(41 + i).standard_normal(om.n_nodes)
    mask = O.dirichlet_mask(om)
    for tr in (False, True):
        At = A.T.tocsr() if tr else A
        y = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.apply(0, _dev(x), y, "fp64", tr)
        yv = y.cpu().numpy()
        assert rel_err(yv, At @ x) < 1e-13, tr
        assert rowwise_excess(yv, At @ x, B.T.tocsr() if tr else B, x, 80, U64) <= 1.0, tr
        assert np.array_equal(yv[mask], x[mask])
