"""GPU tests of the autograd wrapper (finite-difference gradient check) and of the
request server (continuous batching: results identical alone and in a mix, admission
by footprint, error statuses)."""
import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built, gpu_mesh, mat_dict, parity_rtol, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAT = O.Material(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("spacetime", [False, True])
def test_autograd_gradient_matches_oracle_and_central_differences(spacetime):
    from paper_2508_09589_gb300 import options, source
    from paper_2508_09589_gb300.autograd import objective
    om = O.Mesh((12, 8), 8, mat=MAT, bc="patch_left", bc_width=0.3)
    rng = np.random.default_rng(21)
    g0 = 0.2 + 0.6 * rng.random(om.elem_shape if spacetime else (8, 12))
    gm = gpu_mesh(om, coarse_dof_cap=200)
    src = source("sin_t")
    sol = O.forward(om, g0, "sin_t", 1.0)
    rt = max(1e-14, parity_rtol(sol.A, sol.s, sol.f) / 10)
    opts = options(rtol=rt, precision="fp64", max_it=400)
    g = torch.tensor(g0, dtype=torch.float64, device="cuda", requires_grad=True)
    phi = objective(g, gm, src, opts)
    phi.backward()
    grad = g.grad.cpu().numpy()
    # oracle adjoint gradient
    lam = O.adjoint(sol.A, sol.f, O.dirichlet_mask(om), sol.lu)
    ref = O.sensitivities(om, g0, sol.s, lam, extruded=not spacetime)
    assert rel_err(grad, ref) < 1e-9
    # central differences with step 1e-6 through the same GPU solves
    h = 1e-6
    for flat in rng.choice(g0.size, 6, replace=False):
        idx = np.unravel_index(flat, g0.shape)
        vals = []
        for sgn in (1, -1):
            gp = g0.copy()
            gp[idx] += sgn * h
            with torch.no_grad():
                vals.append(objective(torch.tensor(gp, dtype=torch.float64, device="cuda"), gm, src, opts).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(grad[idx] - fd) <= 1e-5 * abs(grad[idx]) + 1e-12 * abs(phi.item()), (idx, grad[idx], fd)


def _req_set(seed=3):
    rng = np.random.default_rng(seed)
    reqs = []
    for r, (ns, nt) in enumerate([((32, 32), 32), ((48, 32), 32), ((32, 64), 48), ((64, 64), 32), ((32, 32), 64),
                                  ((48, 48), 48)]):
        g = rng.random(tuple(reversed(ns)))
        reqs.append((ns, nt, g))
    return reqs


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_server_results_identical_alone_and_in_mix(precision):
    """Each request alone (one slot, no batching) and in a mix (four slots, batches of up to eight
    requests solved together in shared graph launches): bit-identical results, and the mix did
    put several requests into one batch."""
    from paper_2508_09589_gb300 import Server, options
    reqs = _req_set()
    kw = dict(material=mat_dict(MAT))
    opts = options(rtol=1e-8, precision=precision)
    alone = []
    srv = Server(hbm_budget=40 << 30, max_inflight=1, max_batch=1)
    for ns, nt, g in reqs:
        t = srv.submit(ns, nt, g, opts=opts, **kw)
        alone.append(srv.wait(t))
    srv.close()
    srv = Server(hbm_budget=40 << 30, max_inflight=2, max_batch=8)
    tickets = [srv.submit(ns, nt, g, opts=opts, **kw) for ns, nt, g in reqs]
    mixed = [srv.wait(t) for t in tickets]
    srv.close()
    for (ra, ga), (rm, gm_) in zip(alone, mixed):
        assert ra["status"] == 0 and rm["status"] == 0
        assert ra["batch"] == 1
        assert ra["phi"] == rm["phi"]
        np.testing.assert_array_equal(ga, gm_)
        assert ra["forward"]["outer_its"] == rm["forward"]["outer_its"]
        assert ra["forward"]["rel_res"] <= 1e-8 and ra["adjoint"]["rel_res"] <= 1e-8
    assert max(r["batch"] for r, _ in mixed) >= 2


def test_batched_solves_match_single_solves_and_the_oracle():
    """st_solve_forward_batch / st_solve_adjoint_batch over meshes of different sizes, designs
    and layouts: every state, adjoint and gradient equals the mesh's own st_solve_forward /
    st_solve_adjoint bit for bit, and the oracle within the parity tolerances."""
    from paper_2508_09589_gb300 import options, solve_adjoint_batch, solve_forward_batch
    cases = [((24, 16), 12, False), ((20, 20), 16, True), ((32, 24), 8, False)]
    rng = np.random.default_rng(41)
    meshes, designs, oms = [], [], []
    for ns, nt, st in cases:
        om = O.Mesh(ns, nt, mat=MAT, bc="patch_left", bc_width=0.3)
        g = rng.random(om.elem_shape if st else tuple(reversed(ns)))
        gm = gpu_mesh(om, coarse_dof_cap=200)
        gm.set_design(g)
        meshes.append(gm)
        designs.append(g)
        oms.append(om)
    sols = [O.forward(om, g, "uniform", 1.0) for om, g in zip(oms, designs)]
    rt = max(parity_rtol(sol.A, sol.s, sol.f) for sol in sols)
    opts = options(rtol=rt, precision="mixed", max_it=400)
    fst = solve_forward_batch(meshes, opts=opts)
    phis, ast = solve_adjoint_batch(meshes, opts=opts)
    out = [(gm.state("T"), gm.state("lambda"), gm.sensitivities()) for gm in meshes]
    for k, (gm, g, om) in enumerate(zip(meshes, designs, oms)):
        assert fst[k]["status"] == 0 and fst[k]["converged"] and ast[k]["converged"]
        st1 = gm.solve_forward(opts=opts)
        phi1, sa1 = gm.solve_adjoint(opts=opts)
        assert st1["outer_its"] == fst[k]["outer_its"] and sa1["outer_its"] == ast[k]["outer_its"]
        assert phi1 == phis[k]
        np.testing.assert_array_equal(gm.state("T"), out[k][0])
        np.testing.assert_array_equal(gm.state("lambda"), out[k][1])
        np.testing.assert_array_equal(gm.sensitivities(), out[k][2])
        assert rel_err(out[k][0], sols[k].s) < 1e-10


def test_server_matches_direct_mesh_solve():
    from paper_2508_09589_gb300 import Server, options
    ns, nt, g = _req_set()[1]
    opts = options(rtol=1e-10, precision="mixed")
    srv = Server(hbm_budget=8 << 30, max_inflight=2)
    res, grad = srv.wait(srv.submit(ns, nt, g, opts=opts, material=mat_dict(MAT)))
    srv.close()
    om = O.Mesh(ns, nt, mat=MAT)
    gm = gpu_mesh(om)
    gm.set_design(g)
    gm.solve_forward(opts=opts)
    phi, _ = gm.solve_adjoint("compliance", opts=opts)
    assert res["phi"] == phi
    np.testing.assert_array_equal(grad, gm.sensitivities())


def test_server_admission_and_error_statuses():
    from paper_2508_09589_gb300 import Server, STError, footprint_bytes, options
    ns, nt, g = _req_set()[0]
    fp = footprint_bytes(ns, nt, material=mat_dict(MAT))
    srv = Server(hbm_budget=fp // 2, max_inflight=2)
    with pytest.raises(STError) as e:
        srv.submit(ns, nt, g, material=mat_dict(MAT))
    assert e.value.code == -7  # ST_ERR_BUSY: can never fit
    srv.close()
    srv = Server(hbm_budget=4 << 30, max_inflight=2)
    bad = srv.submit(ns, nt, np.zeros(7), layout="extruded", material=mat_dict(MAT))
    slow = srv.submit(ns, nt, g, opts=options(rtol=1e-14, max_it=1), material=mat_dict(MAT))
    ok = srv.submit(ns, nt, g, material=mat_dict(MAT))
    rb, _ = srv.wait(bad)
    rs, _ = srv.wait(slow)
    ro, _ = srv.wait(ok)
    srv.close()
    assert rb["status"] == -1  # ST_ERR_ARG (design size)
    assert rs["status"] == -3  # ST_ERR_NOT_CONVERGED
    assert ro["status"] == 0 and ro["latency_s"] >= ro["queue_s"] >= 0
