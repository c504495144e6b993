"""Failure paths on the GPU, made without faulting, trapping or hanging it: non-finite inputs
are rejected with a status, a grid-barrier wait of the persistent coarse V-cycle tail is made
to give up by a tiny poll limit (the kernel then reports ST_ERR_TIMEOUT and the context stays
usable), and a queued server request is cancelled on the host."""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built, gpu_mesh, mat_dict, parity_rtol, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAT = O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_design_is_rejected_and_the_mesh_recovers(bad):
    from paper_2508_09589_gb300 import STError
    om = O.Mesh((20, 12), 8, mat=MAT, bc="patch_left", bc_width=0.3)
    g = np.random.default_rng(1).random((12, 20))
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gb = g.copy()
    gb[3, 7] = bad
    with pytest.raises(STError) as e:
        gm.set_design(gb)
    assert e.value.code == -4  # ST_ERR_NUMERIC
    with pytest.raises(STError) as e:
        gm.solve_forward()
    assert e.value.code == -8  # ST_ERR_STATE: no valid design
    # the same mesh accepts a valid design afterwards and solves to the oracle's answer
    gm.set_design(g)
    sol = O.forward(om, g, "uniform", 1.0)
    st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision="fp64", max_it=400)
    assert st["converged"] and rel_err(gm.state("T"), sol.s) < 1e-10


def test_non_finite_source_and_warm_start_state_are_rejected():
    from paper_2508_09589_gb300 import STError
    om = O.Mesh((20, 12), 8, mat=MAT, bc="patch_left", bc_width=0.3)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(np.random.default_rng(2).random((12, 20)))
    for kw in (dict(q0=np.nan), dict(kind="sin_t", b=np.inf), dict(kind="sin_t", f=np.nan)):
        with pytest.raises(STError) as e:
            gm.solve_forward(**kw)
        assert e.value.code == -1  # ST_ERR_ARG
    s = np.zeros(om.n_nodes)
    s[om.n_nodes // 2] = np.nan
    gm.set_state(s)
    with pytest.raises(STError) as e:
        gm.solve_forward(warm_start=True)
    assert e.value.code == -4  # ST_ERR_NUMERIC
    assert gm.solve_forward(rtol=1e-8)["converged"]


def test_persistent_tail_barrier_timeout_reports_and_context_survives(monkeypatch):
    """With the whole V-cycle in the cooperative tail kernel and its barrier waits limited to
    one poll, blocks that arrive early give up: the kernel records it, every block still runs
    to its end (all loops are bounded and every index stays in range whatever the data), and
    the solve returns ST_ERR_TIMEOUT.  The next mesh on the same context solves normally."""
    from paper_2508_09589_gb300 import STError
    om = O.Mesh((36, 20), 16, mat=MAT, bc="patch_bottom", bc_width=0.25)
    g = np.random.default_rng(3).random((20, 36))
    monkeypatch.setenv("ST_VTAIL_NODES", "100000000")
    monkeypatch.setenv("ST_VTAIL_SPIN_LIMIT", "1")
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    with pytest.raises(STError) as e:
        gm.solve_forward(rtol=1e-8, max_it=3)
    assert e.value.code == -5  # ST_ERR_TIMEOUT
    gm.close()
    monkeypatch.delenv("ST_VTAIL_SPIN_LIMIT")
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g)
    sol = O.forward(om, g, "uniform", 1.0)
    st = gm.solve_forward(rtol=parity_rtol(sol.A, sol.s, sol.f), precision="fp64", max_it=400)
    assert st["converged"] and rel_err(gm.state("T"), sol.s) < 1e-10


def test_server_cancels_a_queued_request():
    from paper_2508_09589_gb300 import Server, options
    rng = np.random.default_rng(4)
    ns, nt = (64, 64), 64
    srv = Server(hbm_budget=16 << 30, max_inflight=1)
    first = srv.submit(ns, nt, rng.random((64, 64)), opts=options(rtol=1e-10), material=mat_dict(MAT))
    queued = srv.submit(ns, nt, rng.random((64, 64)), material=mat_dict(MAT))
    assert srv.cancel(queued) == 0
    assert srv.cancel(queued) == -8       # already finished (cancelled)
    res, _ = srv.wait(queued)
    assert res["status"] == -10           # ST_ERR_CANCELLED
    assert srv.cancel(queued) == -9       # released by the poll above
    r1, _ = srv.wait(first)
    assert r1["status"] == 0
    assert srv.cancel(first) == -9
    srv.close()
