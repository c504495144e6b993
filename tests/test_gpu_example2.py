"""Example 2's moving Gaussian source (Sec. 2.3.2) on the GPU: the right-hand side against the
oracle's assembled source (the same 2-point Gauss rule per axis and element), and forward, adjoint
and sensitivities of the all-walls problem in both precisions against the oracle's direct
solution, for a space-time and an extruded design; 3-D meshes and non-positive widths are
refused."""
import math

import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built, gpu_mesh, parity_rtol, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the paper's source: peak 1, width 0.05, radius 0.25, one rotation per 2 units of time
SRC = dict(q0=1.0, a=0.05, b=0.25, f=math.pi)
MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("layout", ["spacetime", "extruded"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_example2_rhs_and_solves(layout, precision):
    om = O.Mesh((40, 36), 24, mat=MAT, bc="all_walls", bc_width=0.1, tau=2.0)
    rng = np.random.default_rng(61)
    g = rng.random(om.elem_shape if layout == "spacetime" else tuple(reversed(om.ns)))
    center = (0.5 * om.ext[0], 0.5 * om.ext[1])
    sol = O.forward(om, g, "gaussian", SRC["q0"], a=SRC["a"], b=SRC["b"], f=SRC["f"], center=center)
    dm = O.dirichlet_mask(om)
    lam = O.adjoint(sol.A, sol.f, dm, sol.lu)
    sens = O.sensitivities(om, g, sol.s, lam, extruded=layout == "extruded")
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g, layout)
    rt = parity_rtol(sol.A, sol.s, sol.f)
    st = gm.solve_forward(rtol=rt, precision=precision, max_it=400, kind="gaussian", **SRC)
    assert st["converged"] and st["rel_res"] <= rt
    np.testing.assert_allclose(gm.state("rhs"), sol.f, rtol=0, atol=1e-14 * np.abs(sol.f).max())
    assert rel_err(gm.state("T"), sol.s) < 1e-10
    phi, sta = gm.solve_adjoint("compliance", rtol=parity_rtol(sol.A.T, lam, sol.f), precision=precision,
                                max_it=400)
    assert sta["converged"]
    np.testing.assert_allclose(phi, O.compliance(sol.f, sol.s), rtol=1e-11)
    assert rel_err(gm.state("lambda"), lam) < 1e-10
    assert rel_err(gm.sensitivities(), sens.reshape(-1)) < 1e-9


def test_example2_source_refused_in_3d_and_without_width():
    from paper_2508_09589_gb300 import _lib as L
    om3 = O.Mesh((6, 4, 8), 6, mat=MAT, bc="all_walls", bc_width=0.1)
    gm3 = gpu_mesh(om3, coarse_dof_cap=300)
    gm3.set_design(np.random.default_rng(1).random(tuple(reversed(om3.ns))), "extruded")
    with pytest.raises(Exception):
        gm3.solve_forward(rtol=1e-8, kind="gaussian", **SRC)
    om = O.Mesh((16, 16), 8, mat=MAT, bc="all_walls", bc_width=0.1)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(np.random.default_rng(2).random(tuple(reversed(om.ns))), "extruded")
    with pytest.raises(Exception):
        gm.solve_forward(rtol=1e-8, kind="gaussian", q0=1.0, a=0.0, b=0.25, f=math.pi)
    assert "width" in L.lib().st_last_error().decode()
