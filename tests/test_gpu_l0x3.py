"""The time-marching kernels of extruded 3-D designs in FP32 (k_l0x3.cu), on level 0 and on the
coarse levels (stencils extracted from the Galerkin blocks): operator apply, smoother apply and
start, residual inside the mixed V-cycle, and mixed solves, against the oracle; and the FP64
outer operator on its marching kernel (k_fg_march.cu). Cases: ragged 16 x 4 x 4 tiles on every
axis, every boundary kind, few time slabs, and thread-block budgets that cut the time axis into
short chunks with a ragged last chunk."""
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
    ((17, 9, 6), 5, "patch_left", 0.4, 0),
    ((16, 8, 8), 4, "patch_bottom", 0.5, 0),
    ((6, 4, 8), 6, "all_walls", 0.1, 0),
    ((4, 6, 4), 3, "none", 0.1, 0),
    ((17, 9, 6), 7, "patch_left", 0.3, 24),
    ((3, 3, 3), 1, "patch_left", 0.5, 0),
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
    g = np.random.default_rng(800 + i).random(tuple(reversed(ns)))
    gm = gpu_mesh(om, coarse_dof_cap=300, march_blocks=blocks)
    gm.set_design(g, "extruded")
    return om, g, gm


@pytest.mark.parametrize("i", range(len(CASES)))
def test_fp32_apply_rowwise(i):
    """y = A x and A^T x in FP32 within c u32 (|J|_elem |x|)_i of the oracle on the BF16 design,
    row by row (c = 280: up to 216 summed terms per 3+1-D row; prescribed rows exact)."""
    om, g, gm = _case(i)
    g16 = bf16_round(g)
    A = O.assemble(om, g16)
    B = O.abs_operator(om, g16)
    x = np.random.default_rng(5 + i).standard_normal(om.n_nodes)
    x32 = x.astype(np.float32).astype(np.float64)
    mask = O.dirichlet_mask(om)
    for tr in (False, True):
        At = A.T.tocsr() if tr else A
        y = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.apply(0, _dev(x, torch.float32), y, "mixed", tr)
        yv = y.cpu().numpy().astype(np.float64)
        assert rowwise_excess(yv, At @ x32, B.T.tocsr() if tr else B, x32, 280, U32) <= 1.0, tr
        assert np.array_equal(yv[mask], x32[mask])


@pytest.mark.parametrize("i", range(len(CASES)))
@pytest.mark.parametrize("zero_init", [True, False])
def test_fp32_smoother(i, zero_init):
    """Jacobi-GMRES(10) at level 0 in FP32: its error against the FP64 oracle stays within 10x
    the error of the oracle's own float32 run on the same inputs."""
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


@pytest.mark.parametrize("i", [1, 2, 3])
def test_mixed_vcycle_and_solves(i):
    """The mixed V-cycle (level-0 residual and post-smoothing start on the marching kernels)
    against the oracle's float32 V-cycle, and mixed / FP64 solves to the oracle's direct
    solution."""
    om, g, gm = _case(i)
    lev = O.hierarchy(om, coarse_cap=300)
    assert len(lev) >= 2
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


@pytest.mark.parametrize("i", [1, 2, 3])
def test_fp32_coarse_apply_rowwise(i):
    """Every coarse level with at least two time slabs (space-, time- and mixed coarsening):
    y = A_l x and A_l^T x in FP32, from the two stencils extracted from the FP64 Galerkin blocks,
    within 280 u32 (B_l |x|)_i of the oracle's P^T A P row by row (B_l the Galerkin products of
    |J|_elem), prescribed rows exact."""
    om, g, gm = _case(i)
    olev = O.hierarchy(om, coarse_cap=300)
    assert [(tuple(L.ns), L.nt, L.to_next) for L in olev] == [(L["ns"], L["nt"], L["to_next"])
                                                             for L in gm.levels()]
    mg = O.build_mg(om, g, olev)
    B = O.abs_operator(om, g)
    rng = np.random.default_rng(21 + i)
    checked = 0
    for l in range(1, len(mg)):
        B = galerkin_abs(B, mg[l - 1].Pt, mg[l].mask)
        if olev[l].nt < 2:
            continue
        N = mg[l].A.shape[0]
        x = rng.standard_normal(N)
        x32 = x.astype(np.float32).astype(np.float64)
        for tr in (False, True):
            A = mg[l].A.T.tocsr() if tr else mg[l].A
            y = torch.empty(N, dtype=torch.float32, device="cuda")
            gm.apply(l, _dev(x, torch.float32), y, "mixed", tr)
            yv = y.cpu().numpy().astype(np.float64)
            assert rowwise_excess(yv, A @ x32, B.T.tocsr() if tr else B, x32, 280, U32) <= 1.0, (l, tr)
            assert np.array_equal(yv[mg[l].mask], x32[mg[l].mask])
        checked += 1
    assert checked >= 1


@pytest.mark.parametrize("i", range(len(CASES)))
def test_fp64_apply_rowwise(i):
    """The FP64 outer operator on the marching kernels (k_fg_march.cu, extruded 3-D): y = J x and
    J^T x from the FP64 design within 280 u64 (|J|_elem |x|)_i of the oracle row by row and 1e-13
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
        assert rowwise_excess(yv, At @ x, B.T.tocsr() if tr else B, x, 280, U64) <= 1.0, tr
        assert np.array_equal(yv[mask], x[mask])
