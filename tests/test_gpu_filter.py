"""GPU parity of the PDE filter, the Heaviside projection and their chain rule (Sec. 3.3.2)
against the FP64 oracle: space-time and extruded fields in 2+1-D and 3+1-D on ragged meshes,
and the gradient of the filtered, projected compliance against the oracle's chain rule and
central differences through the GPU solves."""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import U64, ensure_built, gpu_mesh, parity_rtol, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("ns,nt,spacetime,radii", [((40, 24), 20, True, (0.0, 0.0)), ((36, 20), 16, False, (0.0, 0.0)),
                                                   ((33, 17), 12, True, (0.08, 0.3)), ((6, 4, 8), 6, False, (0.3, 0.0)),
                                                   ((5, 6, 4), 5, True, (0.4, 0.5))])
def test_filter_matches_oracle(ns, nt, spacetime, radii):
    """Radii 0 select the paper's minimum, 2.4 h_min and 2.4 dt; the filtered field matches the
    oracle's direct solve, device and host pointers agree, constants and sums are preserved."""
    om = O.Mesh(ns, nt, mat=MAT, bc="patch_left", bc_width=0.3)
    g = np.random.default_rng(7).random(om.elem_shape if spacetime else tuple(reversed(ns)))
    r_x = radii[0] if radii[0] > 0 else 2.4 * min(om.h)
    r_t = radii[1] if radii[1] > 0 else 2.4 * om.dt
    ref = O.pde_filter(om, g, r_x, r_t)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    out, its = gm.filter(g.reshape(-1), radii[0], radii[1], rtol=1e-14)
    assert its > 0
    assert rel_err(out, ref.reshape(-1)) < 1e-11
    gd = torch.tensor(g.reshape(-1), dtype=torch.float64, device="cuda")
    outd, _ = gm.filter(gd, radii[0], radii[1], rtol=1e-14)
    np.testing.assert_array_equal(outd.cpu().numpy(), out)
    one, _ = gm.filter(np.ones(g.size), radii[0], radii[1], rtol=1e-14)
    np.testing.assert_allclose(one, 1.0, rtol=1e-12)
    np.testing.assert_allclose(out.sum(), g.sum(), rtol=1e-12)


def test_heaviside_matches_oracle():
    """H within a few ulps; H' = beta (1 - tanh^2) / den loses relative accuracy in the tails by
    cancellation (an ulp of difference in tanh near +-1), so it is compared within an absolute
    8 beta u / den of its scale."""
    om = O.Mesh((8, 8), 4, mat=MAT)
    gm = gpu_mesh(om)
    x = np.random.default_rng(8).random(500)
    for beta, eta in ((32.0, 0.5), (8.0, 0.3)):
        h, dh = gm.heaviside(x, beta, eta)
        np.testing.assert_allclose(h, O.heaviside(x, beta, eta), rtol=1e-14, atol=1e-15)
        den = np.tanh(beta * eta) + np.tanh(beta * (1 - eta))
        np.testing.assert_allclose(dh, O.heaviside_derivative(x, beta, eta), rtol=1e-13, atol=8 * beta * U64 / den)


@pytest.mark.parametrize("spacetime", [False, True])
def test_filtered_projected_gradient_matches_oracle_and_central_differences(spacetime):
    from paper_2508_09589_gb300 import options, source
    from paper_2508_09589_gb300.autograd import filter_project, objective
    om = O.Mesh((12, 8), 8, mat=MAT, bc="patch_left", bc_width=0.3)
    rng = np.random.default_rng(9)
    g0 = 0.3 + 0.4 * rng.random(om.elem_shape if spacetime else (8, 12))
    r_x, r_t, beta, eta = 0.25, 0.3, 8.0, 0.5
    gb_ref, gt_ref = O.design_chain(om, g0, r_x, r_t, beta, eta)
    sol = O.forward(om, gb_ref, "uniform", 1.0)
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    dphys = O.sensitivities(om, gb_ref, sol.s, lam, extruded=not spacetime)
    ref = O.chain_rule(om, dphys, gt_ref, r_x, r_t, beta, eta)
    gm = gpu_mesh(om, coarse_dof_cap=200)
    opts = options(rtol=max(1e-14, parity_rtol(sol.A, sol.s, sol.f) / 10), precision="fp64", max_it=400)
    src = source()
    g = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
    phi = objective(filter_project(g, gm, r_x, r_t, beta, eta), gm, src, opts)
    phi.backward()
    grad = g.grad.numpy()
    assert rel_err(grad, ref) < 1e-9
    h = 1e-6
    for flat in rng.choice(g0.size, 4, replace=False):
        idx = np.unravel_index(flat, g0.shape)
        vals = []
        for sgn in (1, -1):
            gp = g0.copy()
            gp[idx] += sgn * h
            with torch.no_grad():
                t = torch.tensor(gp, dtype=torch.float64)
                vals.append(objective(filter_project(t, gm, r_x, r_t, beta, eta), gm, src, opts).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(grad[idx] - fd) <= 1e-5 * abs(grad[idx]) + 1e-10 * abs(phi.item()), (idx, grad[idx], fd)
