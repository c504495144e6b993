"""Pins of the oracle's BDF1 reference solver (Sec. 4) beyond its agreement with the hand-written
backward Euler of the P6 pin: closed forms on insulated domains (the per-step slab design and the
time at which the source is taken are fixed by them), the steady state it must reach, and the
spatial element matrices."""
import math

import numpy as np
import pytest

from oracle import st_oracle as O


@pytest.mark.parametrize("ns", [(6, 5), (3, 4, 2)])
def test_insulated_uniform_heating_is_exact(ns):
    """No sink, a uniform design and a uniform source: T^n = n dt q0 / C at every node (the
    constant field is in the kernel of K and M_C 1 = C M 1)."""
    m = O.Mesh(ns, 5, bc="none", tau=2.0)
    T = O.bdf1_forward(m, np.full(tuple(reversed(ns)), 0.6), "uniform", 1.7)
    C = O.simp_C(m.mat, 0.6)
    exact = np.arange(6)[:, None] * m.dt * 1.7 / C
    np.testing.assert_allclose(T, np.broadcast_to(exact, T.shape), rtol=1e-13, atol=1e-15)


def test_space_time_design_and_source_time_of_each_step():
    """Insulated, per-slab uniform designs and a sine source: step n uses the design of slab n
    and Q(t_{n+1}): T^{n+1} = T^n + dt Q(t_{n+1}) / C_n."""
    m = O.Mesh((4, 3), 6, bc="none", tau=1.5)
    vals = np.array([0.1, 0.9, 0.4, 0.7, 0.2, 1.0])
    g = np.broadcast_to(vals[:, None, None], m.elem_shape).copy()
    T = O.bdf1_forward(m, g, "sin_t", 2.0, a=1.0, b=0.5, f=1.3)
    expect = [0.0]
    for n in range(6):
        t1 = (n + 1) * m.dt
        expect.append(expect[-1] + m.dt * 2.0 * (1.0 + 0.5 * math.sin(2 * math.pi * 1.3 * t1)) /
                      O.simp_C(m.mat, vals[n]))
    np.testing.assert_allclose(T[:, 5], expect, rtol=1e-13)
    assert np.ptp(T, axis=1).max() < 1e-12 * np.abs(T).max()


def test_reaches_the_steady_state():
    """A constant source with a sink: T^n tends to the steady solution K_k T = F (the fixed
    point of the step), here after 300 steps of dt = 1 to 1e-10."""
    m = O.Mesh((3, 3, 3), 300, bc="patch_left", bc_width=0.5, tau=300.0)
    g = np.random.default_rng(4).random((3, 3, 3))
    T = O.bdf1_forward(m, g, "uniform", 1.0)
    Mc, Kk = O.bdf1_matrices(m, g)
    F = O.bdf1_load(m, O.source_fn("uniform", 1.0), 0.0)
    n_sp = F.size
    dm = O.dirichlet_mask(m).reshape(m.nt + 1, n_sp)[1]
    K = Kk.toarray()
    K[dm] = 0
    K[:, dm] = 0
    K[dm, dm] = 1
    F[dm] = 0
    steady = np.linalg.solve(K, F)
    assert np.abs(T[-1] - steady).max() < 1e-10 * np.abs(steady).max()


def test_spatial_element_matrices_closed_forms():
    """Tensor products of the 1-D mass h/6 [[2,1],[1,2]] and stiffness 1/h [[1,-1],[-1,1]]."""
    h = (0.3, 0.7)
    Me, Ke = O.spatial_element_matrices(h)
    m1 = lambda hh: hh / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k1 = lambda hh: np.array([[1.0, -1.0], [-1.0, 1.0]]) / hh
    np.testing.assert_allclose(Me, np.kron(m1(h[1]), m1(h[0])), rtol=1e-14)
    np.testing.assert_allclose(Ke, np.kron(m1(h[1]), k1(h[0])) + np.kron(k1(h[1]), m1(h[0])), rtol=1e-13)


@pytest.mark.parametrize("spacetime", [False, True])
def test_adjoint_sensitivities_match_central_differences(spacetime):
    """d phi / d gamma of bdf1_adjoint (the p-norm of the trajectory's element means) equals central
    differences of phi(gamma) through the whole stepping; a wrong slab in M_m Lambda^{m+1}, a
    missing capacity term or a sign error fails it."""
    m = O.Mesh((4, 3), 5, mat=O.Material(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3),
               bc="patch_left", bc_width=0.5, tau=1.5)
    rng = np.random.default_rng(12)
    g = 0.2 + 0.6 * rng.random(m.elem_shape if spacetime else (3, 4))
    kw = dict(source="sin_t", q0=1.0, a=1.0, b=0.8, f=1.0)
    T = O.bdf1_forward(m, g, **kw)
    phi, lam, sens = O.bdf1_adjoint(m, g, T, P=6)
    assert sens.shape == g.shape
    assert np.all(lam[0] == 0.0)

    def value(gam):
        return O.pnorm(m, O.bdf1_forward(m, gam, **kw).reshape(-1), 6)[0]

    assert value(g) == pytest.approx(phi, rel=1e-14)
    h = 1e-6
    for flat in rng.choice(g.size, 6, replace=False):
        idx = np.unravel_index(flat, g.shape)
        gp, gm_ = g.copy(), g.copy()
        gp[idx] += h
        gm_[idx] -= h
        np.testing.assert_allclose(sens[idx], (value(gp) - value(gm_)) / (2 * h), rtol=1e-6, atol=1e-10 * phi)
