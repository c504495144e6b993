"""The damped Jacobi smoother variant (ST_SMOOTH_JACOBI) on the GPU against the oracle's
Jacobi-smoothed V-cycle: FP64 to 1e-8 and mixed precision within the float32 oracle's own error,
both orientations, 2-D stencil levels and element-block levels (space-time and 3-D designs);
forward, adjoint and sensitivities through FGMRES against the oracle's direct solution; and the
argument checks."""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import U32, ensure_built, gpu_mesh, parity_rtol, rel_err
from tests.test_gpu_parity import FP32_FACTOR, _case, _dev, _mixed_levels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OMEGA = 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("i", [0, 1, 3])
def test_jacobi_vcycle_matches_oracle(i):
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300, smoother="jacobi", smoother_omega=OMEGA)
    gm.set_design(g)
    mg = O.build_mg(om, g, O.hierarchy(om, coarse_cap=300))
    b = np.random.default_rng(4).standard_normal(om.n_nodes)
    b[mg[0].mask] = 0
    for tr in (False, True):
        ref = O.vcycle(mg, b, transpose=tr, smoother="jacobi", omega=OMEGA)
        x = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
        gm.vcycle(_dev(b), x, "fp64", tr)
        assert rel_err(x.cpu().numpy(), ref) < 1e-8, tr
    gm.close()


@pytest.mark.parametrize("i", [0, 1, 3])
def test_mixed_jacobi_vcycle_matches_float32_oracle(i):
    om, g = _case(i)
    gm = gpu_mesh(om, coarse_dof_cap=300, smoother="jacobi", smoother_omega=OMEGA)
    gm.set_design(g)
    mg = _mixed_levels(om, g, O.build_mg(om, g, O.hierarchy(om, coarse_cap=300)))
    b = np.random.default_rng(4).standard_normal(om.n_nodes)
    b[mg[0].mask] = 0
    b32 = b.astype(np.float32).astype(np.float64)
    for tr in (False, True):
        ref = O.vcycle(mg, b32, transpose=tr, smoother="jacobi", omega=OMEGA)
        emu = O.vcycle(mg, b32, transpose=tr, dtype=np.float32, smoother="jacobi", omega=OMEGA)
        x = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
        gm.vcycle(_dev(b, torch.float32), x, "mixed", tr)
        e_gpu, e_emu = rel_err(x.cpu().numpy(), ref), rel_err(emu, ref)
        assert e_gpu <= max(FP32_FACTOR * e_emu, 64 * U32) and e_gpu < 5e-3, (tr, e_gpu, e_emu)
    gm.close()


@pytest.mark.parametrize("i", [0, 2, 3])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_jacobi_smoothed_solves_match_the_direct_solution(i, precision):
    om, g = _case(i)
    sol = O.forward(om, g, "uniform", 1.0)
    dm = O.dirichlet_mask(om)
    lam = O.adjoint(sol.A, sol.f, dm, sol.lu)
    sens = O.sensitivities(om, g, sol.s, lam, extruded=g.size == int(np.prod(om.ns)))
    gm = gpu_mesh(om, coarse_dof_cap=300, smoother="jacobi", smoother_omega=OMEGA)
    gm.set_design(g)
    rt = parity_rtol(sol.A, sol.s, sol.f)
    st = gm.solve_forward(rtol=rt, precision=precision, max_it=600, smooth_steps=2)
    assert st["converged"] and st["rel_res"] <= rt
    assert rel_err(gm.state("T"), sol.s) < 1e-10
    phi, sta = gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision=precision,
                                max_it=600, smooth_steps=2)
    assert sta["converged"]
    assert rel_err(gm.state("lambda"), lam) < 1e-10
    assert rel_err(gm.sensitivities(), sens.reshape(-1)) < 1e-9
    gm.close()


def test_jacobi_arguments():
    from paper_2508_09589_gb300 import Mesh, _lib as L
    for bad in (0.0, 1.5, float("nan")):
        with pytest.raises(L.STError):
            Mesh((8, 8), 4, smoother="jacobi", smoother_omega=bad)
    import ctypes as C
    d = L.MeshDesc()
    L.lib().st_mesh_desc_default(C.byref(d))
    assert d.smoother == 0 and d.smoother_omega == 0.5
    d.smoother = 2
    h = C.c_void_p()
    assert L.lib().st_create_mesh(C.byref(d), C.byref(h)) == -1
