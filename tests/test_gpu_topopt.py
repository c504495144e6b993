"""The design loop on the device (st_topopt_*, Sec. 3.3) against the oracle's design iteration:
iteration by iteration from the GPU's own designs (objective, constraint, the gradients MMA
receives and the next design), for an extruded and a space-time design and for Example 2's
all-walls problem with the moving Gaussian source, and for an extruded 3-D design; a longer run on a
larger mesh that must meet the volume constraint and beat the homogeneous design; and the
argument and state checks."""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built, gpu_mesh, parity_rtol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


# Example 2 (Sec. 2.3.2): all walls cold, the moving Gaussian source, a space-time design
EX2 = dict(q0=1.0, a=0.05, b=0.25, f=math.pi)


@pytest.mark.parametrize("layout,precision,example",
                         [("extruded", "mixed", 1), ("spacetime", "mixed", 1), ("extruded", "fp64", 1),
                          ("spacetime", "mixed", 2), ("extruded", "mixed", 3)])
def test_design_iterations_match_the_oracle(layout, precision, example):
    from paper_2508_09589_gb300 import TopOpt
    if example == 1:
        om = O.Mesh((24, 20), 12, mat=MAT, bc="patch_left", bc_width=0.1, tau=20.0)
        src_o, src_g = dict(source="uniform", q0=1.0), dict(kind="uniform", q0=1.0)
    elif example == 3:  # 3+1-D: an extruded design on a 3-D spatial mesh
        om = O.Mesh((8, 6, 6), 6, mat=MAT, bc="patch_left", bc_width=0.3, tau=5.0)
        src_o, src_g = dict(source="uniform", q0=1.0), dict(kind="uniform", q0=1.0)
    else:
        om = O.Mesh((24, 24), 12, mat=MAT, bc="all_walls", bc_width=0.1, tau=2.0)
        src_o = dict(source="gaussian", center=(0.5, 0.5), **EX2)
        src_g = dict(kind="gaussian", **EX2)
    vf, r_x, r_t = 0.3, 2.4 / om.ns[1], 2.4 * om.tau / om.nt
    shape = tuple(reversed(om.ns)) if layout == "extruded" else om.elem_shape
    g0 = np.full(shape, 0.5)
    g0 += 0.05 * np.random.default_rng(5).standard_normal(shape)  # break the symmetry a little
    sol0 = O.forward(om, np.clip(g0, 0, 1), **src_o)
    rt = parity_rtol(sol0.A, sol0.s, sol0.f)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    to = TopOpt(gm, g0, layout, vf=vf, r_x=r_x, r_t=r_t, filter_rtol=1e-13)
    hist = O.TopOptHistory()
    g = np.clip(g0, 0.0, 1.0)
    np.testing.assert_array_equal(to.get("gamma"), g)
    for it in range(1, 5):
        st = to.step(rtol=rt, precision=precision, max_it=400, allow_not_converged=True, **src_g)
        assert st["forward"]["rel_res"] <= 10 * rt and st["adjoint"]["rel_res"] <= 10 * rt
        g_next, d = O.topopt_step(om, g, hist, vf, r_x, r_t, **src_o)
        assert st["iteration"] == it
        np.testing.assert_allclose(st["phi"], d["phi"], rtol=1e-9)
        assert abs(st["chi"] - d["chi"]) < 1e-10
        np.testing.assert_allclose(to.get("gamma_bar"), d["gamma_bar"], rtol=0, atol=1e-10)
        dphi = to.get("dphi").reshape(-1)
        assert np.abs(dphi - d["df0"]).max() < 1e-8 * np.abs(d["df0"]).max()
        dchi = to.get("dchi").reshape(-1)
        assert np.abs(dchi - d["dchi"].reshape(-1)).max() < 1e-10 * np.abs(d["dchi"]).max()
        assert abs(st["lam"] - d["lam_mma"]) <= 1e-7 * max(abs(d["lam_mma"]), 1.0)
        gg = to.get("gamma")
        assert np.abs(gg - g_next).max() < 1e-7, it
        np.testing.assert_allclose(st["change"], np.abs(gg - g).max(), rtol=0, atol=1e-15)
        g = gg  # the oracle continues from the GPU's design
    to.close()
    gm.close()


def test_design_loop_meets_the_volume_and_beats_the_homogeneous_design():
    """Thirty iterations on a 64 x 64 x 32 space-time mesh with the paper's beta, P and warm-started
    mixed-precision solves: a feasible design whose p-norm temperature is below half that of the
    homogeneous physical design of the same volume."""
    from paper_2508_09589_gb300 import Mesh, TopOpt
    kw = dict(tau=20.0, material=dict(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3),
              bc="patch_left", bc_width=0.1)
    gm = Mesh((64, 64), 32, **kw)
    to = TopOpt(gm, np.full((64, 64), 0.5), vf=0.3)
    chis, phis = [], []
    for _ in range(30):
        st = to.step(rtol=1e-8, max_it=200)
        chis.append(st["chi"])
        phis.append(st["phi"])
        assert st["forward"]["converged"] and st["adjoint"]["converged"]
    g = to.get("gamma")
    assert g.min() >= 0.0 and g.max() <= 1.0
    gb = to.get("gamma_bar")
    assert gb.mean() / 0.3 - 1.0 <= 2e-3
    to.close()
    hom = Mesh((64, 64), 32, **kw)
    hom.set_design(np.full((64, 64), 0.3), "extruded")
    hom.solve_forward(rtol=1e-8, max_it=200)
    phi_hom, _ = hom.solve_adjoint("pnorm", P=20, rtol=1e-8, max_it=200)
    opt = Mesh((64, 64), 32, **kw)
    opt.set_design(gb, "extruded")
    opt.solve_forward(rtol=1e-8, max_it=200)
    phi_opt, _ = opt.solve_adjoint("pnorm", P=20, rtol=1e-8, max_it=200)
    assert phi_opt < 0.5 * phi_hom, (phi_opt, phi_hom, phis[-5:], chis[-5:])


def test_design_loop_arguments_and_state():
    from paper_2508_09589_gb300 import Mesh, TopOpt, _lib as L
    gm = Mesh((8, 8), 4)
    with pytest.raises(L.STError):
        TopOpt(gm, np.full((8, 8), 0.5), vf=1.0)
    with pytest.raises(L.STError):
        TopOpt(gm, np.full((8, 8), 0.5), eta=0.0)
    bad = np.full((8, 8), 0.5)
    bad[2, 3] = np.nan
    with pytest.raises(L.STError) as e:
        TopOpt(gm, bad)
    assert e.value.code == -4
    h = C.c_void_p()
    p = L.TopOptParams()
    L.lib().st_topopt_params_default(C.byref(p))
    g = np.full(63, 0.5)
    assert L.lib().st_topopt_create(gm._h, C.byref(p), C.c_void_p(g.ctypes.data), 0, 63, 0, C.byref(h)) == -1
    to = TopOpt(gm, np.full((8, 8), 1.5))
    np.testing.assert_array_equal(to.get("gamma"), np.ones((8, 8)))  # clipped
    with pytest.raises(L.STError) as e:
        to.get("gamma_bar")
    assert e.value.code == -8
    st = to.step(rtol=1e-8)
    assert st["iteration"] == 1 and st["chi"] > 0
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    to.get("gamma", out=out)
    np.testing.assert_array_equal(out.cpu().numpy().reshape(8, 8), to.get("gamma"))
    to.close()
