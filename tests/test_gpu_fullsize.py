"""Full-size checks on the three solve configurations, in the launch configuration the
benchmark uses (default hierarchy, mixed precision, outer tolerance 1e-8):

* 256^2 x 256 elements, time-constant random-field design (16,974,593 DOFs),
* 512^2 x 256, one density per space-time element, q(t) = 1 + 0.5 sin(8 pi t) (67,634,433),
* 64^3 x 64 in 3-D space, capacity varied by SIMP p_c = 1 (17,850,625).

The oracle cannot assemble or solve these, so it computes sampled outputs one by one:
operator rows (element by element) on a seeded random vector, and source rows.  Solutions
are then checked through properties that hold at any size: the true residual with the
(row-verified) FP64 operator, adjoint duality f^T s = lambda^T f, and a directional central
difference of the compliance against g^T v.
"""
import numpy as np
import pytest

import workloads as W
from oracle import st_oracle as O
from tests.gpu_common import bf16_round, ensure_built

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

CONFIGS = [W.C1.name, W.C2.name, W.C3.name]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


def _setup(name):
    from paper_2508_09589_gb300 import Mesh
    w = W.WORKLOADS[name]
    om = O.Mesh(w.ns, w.nt, mat=O.Material(**w.material), bc=w.bc, bc_width=w.bc_width, tau=w.tau)
    g = W.make_design(w)
    gm = Mesh(w.ns, w.nt, material=w.material, bc=w.bc, bc_width=w.bc_width, tau=w.tau)
    layout = "extruded" if w.extruded else "spacetime"
    gm.set_design(g.reshape(-1), layout)
    return w, om, g, gm, layout


def _sample_rows(om, rng, n=240):
    """Random nodes plus the first, second, last and second-to-last time planes, the
    prescribed patch, and the ragged far edges of every axis."""
    shape = om.node_shape  # (t, [z], y, x)
    N = om.n_nodes
    rows = list(rng.integers(0, N, n))
    for t in (0, 1, 2, shape[0] - 2, shape[0] - 1):
        for _ in range(8):
            idx = [t] + [int(rng.integers(0, s)) for s in shape[1:]]
            rows.append(np.ravel_multi_index(tuple(idx), shape))
    dm = O.dirichlet_mask(om)
    pres = np.flatnonzero(dm[: int(np.prod(shape[1:])) * 3])  # prescribed nodes of the first planes
    rows += list(rng.choice(pres, 8, replace=False))
    for ax in range(1, len(shape)):
        for _ in range(6):
            idx = [int(rng.integers(0, s)) for s in shape]
            idx[ax] = shape[ax] - 1
            rows.append(np.ravel_multi_index(tuple(idx), shape))
    return np.unique(np.asarray(rows, dtype=np.int64))


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", CONFIGS)
def test_fullsize_operator_and_source_rows(name):
    w, om, g, gm, layout = _setup(name)
    rng = np.random.default_rng(21)
    rows = _sample_rows(om, rng)
    x = rng.standard_normal(om.n_nodes)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    for tr in (False,):
        gm.apply(0, xd, y, "fp64", tr)
    ref = O.apply_rows(om, g, x, rows)
    assert _rel(y.cpu().numpy()[rows], ref) < 1e-12
    # FP32 operator of the mixed V-cycle: 27-point FP32 stencils from the FP64 design on
    # time-constant 2-D designs, else the BF16 design
    g32 = g if (w.extruded and om.sd == 2) else bf16_round(g)
    x32 = x.astype(np.float32)
    y32 = torch.empty(om.n_nodes, dtype=torch.float32, device="cuda")
    gm.apply(0, torch.from_numpy(x32).cuda(), y32, "mixed")
    ref32 = O.apply_rows(om, g32, x32.astype(np.float64), rows)
    assert _rel(y32.cpu().numpy()[rows].astype(np.float64), ref32) < 1e-4
    # row by row within the componentwise rounding bound c u32 (|J|_elem |x|)_i
    bnd = O.apply_rows(om, g32, x32.astype(np.float64), rows, absolute=True)
    c = 80 if om.sd == 2 else 280
    err = np.abs(y32.cpu().numpy()[rows].astype(np.float64) - ref32)
    assert (err <= c * 2.0 ** -24 * bnd + 1e-300).all()
    # source vector, assembled on the device at the forward solve
    src = dict(kind=w.source, q0=w.source_q0, a=w.source_a, b=w.source_b, f=w.source_f)
    gm.solve_forward(rtol=1e-2, max_it=3, allow_not_converged=True, **src)
    f = gm.state("rhs")
    fr = O.source_rows(om, O.source_fn(w.source, w.source_q0, w.source_a, w.source_b, w.source_f), rows)
    np.testing.assert_allclose(f[rows], fr, rtol=1e-13, atol=1e-15 * np.abs(fr).max())
    gm.close()


@pytest.mark.parametrize("name", CONFIGS)
def test_fullsize_solves_residual_duality_and_directional_derivative(name):
    w, om, g, gm, layout = _setup(name)
    src = dict(kind=w.source, q0=w.source_q0, a=w.source_a, b=w.source_b, f=w.source_f)
    # the benchmark's solves: mixed precision to 1e-8
    st = gm.solve_forward(rtol=1e-8, max_it=400, **src)
    assert st["converged"] and st["rel_res"] <= 1e-8
    s = gm.state("T")
    f = gm.state("rhs")
    y = torch.empty(om.n_nodes, dtype=torch.float64, device="cuda")
    gm.apply(0, torch.from_numpy(s).cuda(), y, "fp64")
    r = f - y.cpu().numpy()
    assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(f)
    phi, sa = gm.solve_adjoint("compliance", rtol=1e-8, max_it=400)
    assert sa["converged"]
    lam = gm.state("lambda")
    assert abs(float(f @ s) - float(lam @ f)) <= 1e-6 * abs(phi)
    np.testing.assert_allclose(phi, float(f @ s), rtol=1e-12)
    # directional derivative along v = gamma (1 - gamma) (smooth, zero at the bounds) by
    # central differences of tightly solved compliances, against g^T v.  At these sizes the
    # FP64 residual floor is near 1e-12, so the solves aim at 1e-11 and must reach 1e-10:
    # with h = 1e-4 the compliance changes by about 1e-5 relative, far above that noise.
    tight = dict(rtol=1e-11, max_it=300, allow_not_converged=True)
    assert gm.solve_forward(**tight, **src)["rel_res"] < 1e-10
    assert gm.solve_adjoint("compliance", **tight)[1]["rel_res"] < 1e-10
    grad = gm.sensitivities()
    v = (g * (1.0 - g)).reshape(-1)
    gv = float(grad @ v)
    h = 1e-4
    phis = []
    for sgn in (1.0, -1.0):
        gm.set_design((g.reshape(-1) + sgn * h * v), layout)
        assert gm.solve_forward(**tight, **src)["rel_res"] < 1e-10
        fs = gm.state("rhs")
        phis.append(float(fs @ gm.state("T")))
    fd = (phis[0] - phis[1]) / (2 * h)
    assert abs(fd - gv) <= 1e-5 * abs(gv), (fd, gv)
    gm.close()
