"""Pins of the oracle's design iteration (Sec. 3.3): the gradients it hands to MMA against
central differences of the whole chain (filter, projection, state solve, p-norm objective,
volume constraint), and the loop itself against what an optimiser must achieve: a design that
meets the volume constraint and beats the homogeneous design of the same volume."""
import numpy as np
import pytest

from oracle import st_oracle as O

MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@pytest.mark.parametrize("spacetime", [False, True])
def test_design_iteration_gradients_match_central_differences(spacetime):
    """d phi / d gamma and d chi / d gamma of topopt_gradients equal central differences of
    phi(gamma) and chi(gamma) computed through the whole chain; a dropped H' factor, a missing
    filter pass or a wrong adjoint right-hand side of the p-norm fails it."""
    m = O.Mesh((4, 3), 4, mat=MAT, bc="patch_left", bc_width=0.5, tau=2.0)
    rng = np.random.default_rng(71)
    shape = m.elem_shape if spacetime else (3, 4)
    g = 0.35 + 0.3 * rng.random(shape)
    kw = dict(beta=8.0, eta=0.5, P=8)
    r_x, r_t, vf = 0.6, 0.8, 0.4
    d = O.topopt_gradients(m, g, vf, r_x, r_t, **kw)

    def values(gam):
        e = O.topopt_gradients(m, gam, vf, r_x, r_t, **kw)
        return e["phi"], e["chi"]

    h = 1e-6
    for flat in rng.choice(g.size, 6, replace=False):
        idx = np.unravel_index(flat, g.shape)
        gp, gm_ = g.copy(), g.copy()
        gp[idx] += h
        gm_[idx] -= h
        (pp, cp), (pm, cm) = values(gp), values(gm_)
        np.testing.assert_allclose(d["dphi"][idx], (pp - pm) / (2 * h), rtol=1e-5, atol=1e-9 * abs(d["phi"]))
        np.testing.assert_allclose(d["dchi"][idx], (cp - cm) / (2 * h), rtol=1e-5, atol=1e-9)


def test_volume_constraint_is_the_space_time_volume_fraction():
    """chi = 0 exactly at a physical design of mean v_f; its gradient sums to 1 / v_f."""
    g = np.full((3, 5, 6), 0.25)
    chi, dchi = O.volume_constraint(g, 0.25)
    assert chi == 0.0 and dchi.shape == g.shape
    np.testing.assert_allclose(dchi.sum(), 4.0)


def test_design_loop_meets_the_volume_and_beats_the_homogeneous_design():
    """Forty iterations with the paper's beta = 32 and P = 20 from the homogeneous design gamma =
    eta: the design is feasible, lies in [0, 1], and its p-norm temperature is below half that
    of the homogeneous physical design of the same volume (the optimum is a conducting tree).
    The first iteration's MMA gradient is the chain-ruled objective gradient scaled by 10 / phi_1."""
    m = O.Mesh((16, 16), 8, mat=MAT, bc="patch_left", bc_width=0.1, tau=20.0)
    vf, r_x, r_t = 0.3, 2.4 / 16, 2.4 * 20.0 / 8
    g = np.full((16, 16), 0.5)
    hist = O.TopOptHistory()
    g1, d1 = O.topopt_step(m, g, hist, vf, r_x, r_t)
    np.testing.assert_allclose(d1["df0"], 10.0 / d1["phi"] * d1["dphi"].reshape(-1), rtol=1e-15)
    assert hist.phi1 == d1["phi"] and hist.it == 1
    g = g1
    for _ in range(39):
        g, d = O.topopt_step(m, g, hist, vf, r_x, r_t)
    gb, _ = O.design_chain(m, g, r_x, r_t)
    chi, _ = O.volume_constraint(gb, vf)
    assert chi <= 1e-3
    assert g.min() >= 0.0 and g.max() <= 1.0
    sol = O.forward(m, gb, "uniform", 1.0)
    phi_opt = O.pnorm(m, sol.s, 20)[0]
    hom = O.forward(m, np.full((16, 16), vf), "uniform", 1.0)
    phi_hom = O.pnorm(m, hom.s, 20)[0]
    assert phi_opt < 0.5 * phi_hom, (phi_opt, phi_hom)


def test_example2_time_varying_design_beats_the_extruded_one():
    """Example 2 (Sec. 2.3.2; all walls cold, a Gaussian source circling the centre): forty
    iterations from gamma = eta.  Both designs meet the volume and beat the homogeneous design;
    the space-time design, free to move its material with the source, reaches a p-norm
    temperature below a fifth of the extruded design's (the oracle gives 0.0076 against 0.038)."""
    import math
    m = O.Mesh((16, 16), 16, mat=MAT, bc="all_walls", bc_width=0.1, tau=2.0)
    src = dict(source="gaussian", q0=1.0, a=0.05, b=0.25, f=math.pi, center=(0.5, 0.5))
    vf, r_x, r_t = 0.3, 2.4 / 16, 2.4 * 2.0 / 16
    phi_hom = O.pnorm(m, O.forward(m, np.full((16, 16), vf), **src).s, 20)[0]
    phi = {}
    for layout, shape in (("extruded", (16, 16)), ("spacetime", m.elem_shape)):
        g = np.full(shape, 0.5)
        hist = O.TopOptHistory()
        for _ in range(40):
            g, _d = O.topopt_step(m, g, hist, vf, r_x, r_t, **src)
        gb, _ = O.design_chain(m, g, r_x, r_t)
        assert O.volume_constraint(gb, vf)[0] <= 1e-3
        phi[layout] = O.pnorm(m, O.forward(m, gb, **src).s, 20)[0]
    assert phi["extruded"] < 0.5 * phi_hom, (phi, phi_hom)
    assert phi["spacetime"] < 0.2 * phi["extruded"], (phi, phi_hom)
