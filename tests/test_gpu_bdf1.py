"""The time-stepping reference solver on the device (st_bdf1_*, Sec. 4) against the oracle's
BDF1 (direct solve per step): whole trajectories for extruded and space-time designs, 2-D and
3-D, uniform and sine sources, both multigrid precisions; the discrete adjoint and the design
sensitivities of the p-norm; the gap to the all-at-once solution as
dt shrinks; argument and state checks."""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built, gpu_mesh, mat_dict, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


def _bdf1(om, **kw):
    from paper_2508_09589_gb300 import BDF1
    return BDF1(om.ns, om.nt, ext=om.ext, tau=om.tau, material=mat_dict(om.mat), bc=om.bc,
                bc_width=om.bc_width, **kw)


CASES = [
    ((40, 36), 12, "extruded", "uniform", "mixed"),
    ((40, 36), 12, "extruded", "sin_t", "fp64"),
    ((33, 20), 10, "spacetime", "sin_t", "mixed"),
    ((10, 8, 6), 8, "extruded", "uniform", "mixed"),
    ((10, 8, 6), 6, "spacetime", "uniform", "fp64"),
]


@pytest.mark.parametrize("ns,nt,layout,kind,precision", CASES)
def test_trajectory_matches_the_oracle(ns, nt, layout, kind, precision):
    om = O.Mesh(ns, nt, mat=MAT, bc="patch_left", bc_width=0.3, tau=1.0)
    rng = np.random.default_rng(sum(ns) + nt)
    g = rng.random(tuple(reversed(ns)) if layout == "extruded" else om.elem_shape)
    src = dict(q0=1.0, a=1.0, b=0.5, f=2.0) if kind == "sin_t" else dict(q0=1.0)
    ref = O.bdf1_forward(om, g, kind, **src)
    b = _bdf1(om, coarse_dof_cap=300)
    b.set_design(g, layout)
    T, st = b.forward(kind=kind, rtol=1e-13, precision=precision, max_it=300, **src)
    assert st["steps"] == nt and st["max_rel_res"] <= 1e-13
    assert T.shape == ref.shape[:1] + tuple(n + 1 for n in reversed(ns))
    assert rel_err(T.reshape(ref.shape), ref) < 1e-10
    # into a device buffer as well
    out = torch.empty(ref.size, dtype=torch.float64, device="cuda")
    b.forward(kind=kind, rtol=1e-13, precision=precision, max_it=300, out=out, **src)
    assert rel_err(out.cpu().numpy().reshape(ref.shape), ref) < 1e-10
    b.close()


ADJ_CASES = [
    ((30, 26), 10, "extruded", "mixed"),
    ((30, 26), 8, "spacetime", "fp64"),
    ((8, 6, 6), 6, "extruded", "mixed"),
    ((8, 6, 6), 5, "spacetime", "mixed"),
]


@pytest.mark.parametrize("ns,nt,layout,precision", ADJ_CASES)
def test_adjoint_and_sensitivities_match_the_oracle(ns, nt, layout, precision):
    om = O.Mesh(ns, nt, mat=MAT, bc="patch_left", bc_width=0.3, tau=1.0)
    rng = np.random.default_rng(7 * nt + len(ns))
    g = 0.1 + 0.8 * rng.random(tuple(reversed(ns)) if layout == "extruded" else om.elem_shape)
    src = dict(q0=1.0, a=1.0, b=0.5, f=2.0)
    T_ref = O.bdf1_forward(om, g, "sin_t", **src)
    phi_ref, lam_ref, sens_ref = O.bdf1_adjoint(om, g, T_ref, P=20)
    b = _bdf1(om, coarse_dof_cap=300)
    b.set_design(g, layout)
    b.forward(kind="sin_t", rtol=1e-13, precision=precision, max_it=300, **src)
    phi, lam, st = b.adjoint(P=20, rtol=1e-13, precision=precision, max_it=300)
    assert st["steps"] == nt and st["max_rel_res"] <= 1e-13
    np.testing.assert_allclose(phi, phi_ref, rtol=1e-11)
    assert rel_err(lam.reshape(lam_ref.shape), lam_ref) < 1e-9
    sens = b.sensitivities()
    assert rel_err(sens, sens_ref.reshape(-1)) < 1e-9
    out = torch.empty(sens.size, dtype=torch.float64, device="cuda")
    b.sensitivities(out)
    np.testing.assert_array_equal(out.cpu().numpy(), sens)
    b.close()


def test_gap_to_the_all_at_once_solution_shrinks_with_dt():
    """For a time-constant design the all-at-once and the BDF1 trajectories on the same mesh differ
    (the space-time scheme couples time non-causally) by a gap that shrinks as dt is halved; the
    initial layer of the suddenly switched-on source keeps it below first order at these sizes.
    The gaps equal the oracle's (direct solves of both schemes)."""
    gaps, ref = [], []
    g = np.random.default_rng(9).random((24, 24))
    for nt in (16, 32, 64):
        om = O.Mesh((24, 24), nt, mat=MAT, bc="patch_left", bc_width=0.3)
        gm = gpu_mesh(om, coarse_dof_cap=300)
        gm.set_design(g, "extruded")
        gm.solve_forward(rtol=1e-12, max_it=300)
        Ts = gm.state("T").reshape((nt + 1, 25, 25))
        b = _bdf1(om, coarse_dof_cap=300)
        b.set_design(g, "extruded")
        Tb, _ = b.forward(rtol=1e-12, max_it=300)
        gaps.append(np.abs(Ts[:nt] - Tb[:nt]).max())
        ref.append(np.abs(O.forward(om, g).s.reshape(nt + 1, -1)[:nt] - O.bdf1_forward(om, g)[:nt]).max())
        gm.close()
        b.close()
    np.testing.assert_allclose(gaps, ref, rtol=1e-6)
    assert gaps[1] < 0.8 * gaps[0] and gaps[2] < 0.8 * gaps[1]


def test_arguments_and_state():
    from paper_2508_09589_gb300 import BDF1, _lib as L
    b = BDF1((8, 8), 4)
    with pytest.raises(L.STError) as e:
        b.forward()
    assert e.value.code == -8
    with pytest.raises(L.STError):
        b.set_design(np.full(63, 0.5), "extruded")
    bad = np.full((8, 8), 0.5)
    bad[1, 1] = np.inf
    with pytest.raises(L.STError) as e:
        b.set_design(bad)
    assert e.value.code == -4
    b.set_design(np.full((8, 8), 0.5))
    with pytest.raises(L.STError) as e:
        b.forward(kind="gaussian", a=0.05, b=0.25, f=3.0)
    assert e.value.code == -1
    with pytest.raises(L.STError) as e:
        b.adjoint()
    assert e.value.code == -8
    T, st = b.forward(rtol=1e-10)
    assert st["steps"] == 4 and np.all(T[0] == 0.0) and T[-1].max() > 0
    with pytest.raises(L.STError) as e:
        b.sensitivities()
    assert e.value.code == -8
    with pytest.raises(L.STError):
        b.adjoint(P=0)
    phi, lam, _ = b.adjoint(P=4, rtol=1e-10)
    assert phi > 0 and np.all(lam[0] == 0.0)
    assert b.sensitivities().shape == (64,)
    b.close()
