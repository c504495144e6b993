"""The device MMA (st_mma_*, k_mma.cu) against the oracle's MMA (Sec. 3.3.3): iteration by
iteration on the same inputs (asymptotes, subproblem and dual multiplier), convergence to the
closed-form optimum of a separable convex problem, a large random problem from an infeasible
start (capped multiplier), and the argument checks."""
import ctypes as C

import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    assert torch.cuda.is_available()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _lockstep(c, V, iters, xmin=1e-3):
    """GPU and oracle MMA on min sum c / x s.t. mean(x) <= V, each iteration from the GPU's x."""
    from paper_2508_09589_gb300 import MMA
    n = c.size
    mma = MMA(n)
    xg = _dev(np.full(n, V))
    xo1 = xo2 = low = upp = np.zeros(n)
    worst = 0.0
    for it in range(1, iters + 1):
        x = xg.cpu().numpy()
        f0 = np.sum(c / x)
        df0 = -c / x ** 2 / f0
        g1 = x.mean() / V - 1.0
        dg1 = np.full(n, 1.0 / (n * V))
        xo, low, upp, lam_o = O.mma_update(it, x, xo1, xo2, low, upp, df0, g1, dg1, xmin=xmin, xmax=1.0)
        lam_g = mma.update(xg, _dev(df0), g1, _dev(dg1), xmin=xmin, xmax=1.0)
        torch.cuda.synchronize()
        xn = xg.cpu().numpy()
        worst = max(worst, float(np.abs(xn - xo).max()))
        assert abs(lam_g - lam_o) <= 1e-9 * max(abs(lam_o), 1e-300) or lam_g == lam_o == 0.0, (it, lam_g, lam_o)
        xo2, xo1 = xo1, x
    mma.close()
    return xg.cpu().numpy(), worst


def test_mma_matches_the_oracle_iteration_by_iteration_and_converges():
    c = np.random.default_rng(0).random(400) + 0.1
    V = 0.3
    x, worst = _lockstep(c, V, 40)
    assert worst < 1e-12
    exact = V * c.size * np.sqrt(c) / np.sqrt(c).sum()
    assert np.abs(x - exact).max() < 1e-11


def test_mma_large_random_problem_from_an_infeasible_start():
    """A million variables, random objective gradients, a constraint violated beyond what the
    move limits allow at first: the first steps cap the multiplier, later ones find its root;
    every step equals the oracle's."""
    from paper_2508_09589_gb300 import MMA
    rng = np.random.default_rng(1)
    n = 1_000_000
    w = rng.random(n) + 0.5
    x = rng.uniform(0.6, 0.9, n)
    mma = MMA(n)
    xg = _dev(x)
    xo1 = xo2 = low = upp = np.zeros(n)
    lams = []
    for it in range(1, 23):  # the constraint becomes reachable at the 20th step
        x = xg.cpu().numpy()
        df0 = -w * (1.0 - x) / n  # the objective favours larger x
        g1 = x.mean() / 0.4 - 1.0
        dg1 = np.full(n, 1.0 / (n * 0.4))
        xo, low, upp, lam_o = O.mma_update(it, x, xo1, xo2, low, upp, df0, g1, dg1)
        lam_g = mma.update(xg, _dev(df0), g1, _dev(dg1))
        torch.cuda.synchronize()
        assert np.abs(xg.cpu().numpy() - xo).max() < 1e-12, it
        assert abs(lam_g - lam_o) <= 1e-9 * lam_o or lam_g == lam_o == 0.0
        lams.append(lam_g)
        xo2, xo1 = xo1, x
    assert lams[0] >= 1e39 and lams[-1] < 1e39
    mma.close()


def test_mma_arguments():
    from paper_2508_09589_gb300 import _lib as L
    h = C.c_void_p()
    assert L.lib().st_mma_create(0, None, C.byref(h)) == -1
    p = L.MmaParams()
    L.lib().st_mma_params_default(C.byref(p))
    p.decr = 1.5
    assert L.lib().st_mma_create(10, C.byref(p), C.byref(h)) == -1
    assert L.lib().st_mma_create(10, None, C.byref(h)) == 0
    x = _dev(np.full(10, 0.5))
    lam = C.c_double()
    assert L.lib().st_mma_update(h, 0, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 0.0,
                                 C.c_void_p(x.data_ptr()), 0.0, 1.0, None, C.byref(lam)) == -1
    assert L.lib().st_mma_update(h, 1, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), float("nan"),
                                 C.c_void_p(x.data_ptr()), 0.0, 1.0, None, C.byref(lam)) == -1
    assert L.lib().st_mma_destroy(h) == 0
