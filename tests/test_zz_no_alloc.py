"""The allocation-free residual entry point (st_residual_norm_noalloc).

Some callers cannot call cudaMalloc (for example code running inside another framework's
stream capture or fixed memory pool, or a real-time loop).  For them the library offers
r = f - J x and ||r||_2 with all scratch in a static device array.  This test calls it
twice in a row through the C ABI and checks both results against the FP64 oracle's assembled
operator (r = f - A x) and against the regular fine-level operator entry point (st_op_apply),
within the FP64 operator tolerance of the other tests, for both sink-patch placements; and
replays it from a CUDA graph captured on a side stream.
This file sorts last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built, gpu_mesh, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAYOUT = {"extruded": 0, "spacetime": 1}


@pytest.mark.parametrize("bc", ["patch_left", "patch_bottom"])
@pytest.mark.parametrize("ns,nt,layout", [((40, 24), 20, "spacetime"), ((36, 20), 16, "extruded"),
                                          ((6, 4, 8), 6, "extruded")])
def test_residual_norm_noalloc_matches_oracle_and_operator_apply(ns, nt, layout, bc):
    L = ensure_built()
    om = O.Mesh(ns, nt, mat=O.Material(), bc=bc, bc_width=0.3)
    rng = np.random.default_rng(5)
    g = rng.random(om.elem_shape if layout == "spacetime" else tuple(reversed(ns)))
    gm = gpu_mesh(om, coarse_dof_cap=300)
    gm.set_design(g, layout)
    x = torch.tensor(rng.standard_normal(om.n_nodes), dtype=torch.float64, device="cuda")
    f = torch.tensor(rng.standard_normal(om.n_nodes), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    gm.apply(0, x, y, "fp64")
    r_op = (f - y).cpu().numpy()
    A = O.assemble(om, g)
    r_ref = f.cpu().numpy() - A @ x.cpu().numpy()
    n_ref = float(np.linalg.norm(r_ref))
    assert rel_err(r_op, r_ref) < 1e-12
    gd = torch.tensor(np.ascontiguousarray(g).reshape(-1), dtype=torch.float64, device="cuda")
    for _ in range(2):
        r = torch.full_like(x, float("nan"))
        norm = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        code = L.st_residual_norm_noalloc(C.byref(gm.desc), C.c_void_p(gd.data_ptr()), LAYOUT[layout],
                                          C.c_void_p(x.data_ptr()), C.c_void_p(f.data_ptr()),
                                          C.c_void_p(r.data_ptr()), C.c_void_p(norm.data_ptr()), None)
        assert code == 0, L.st_last_error()
        torch.cuda.synchronize()
        assert rel_err(r.cpu().numpy(), r_ref) < 1e-12
        assert rel_err(r.cpu().numpy(), r_op) < 1e-12
        assert abs(norm.item() - n_ref) <= 1e-12 * n_ref


def test_residual_norm_noalloc_captured_in_a_graph():
    """After one eager call on a side stream, the call is captured into a CUDA graph on that
    stream and replayed twice: every replay gives the eager r and norm bit for bit, and both
    match the oracle."""
    L = ensure_built()
    om = O.Mesh((40, 24), 20, mat=O.Material(), bc="patch_left", bc_width=0.3)
    rng = np.random.default_rng(7)
    g = rng.random(om.elem_shape)
    gm = gpu_mesh(om, coarse_dof_cap=300)
    x = torch.tensor(rng.standard_normal(om.n_nodes), dtype=torch.float64, device="cuda")
    f = torch.tensor(rng.standard_normal(om.n_nodes), dtype=torch.float64, device="cuda")
    gd = torch.tensor(np.ascontiguousarray(g).reshape(-1), dtype=torch.float64, device="cuda")
    r = torch.empty_like(x)
    norm = torch.empty(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()

    def call():
        return L.st_residual_norm_noalloc(C.byref(gm.desc), C.c_void_p(gd.data_ptr()), LAYOUT["spacetime"],
                                          C.c_void_p(x.data_ptr()), C.c_void_p(f.data_ptr()),
                                          C.c_void_p(r.data_ptr()), C.c_void_p(norm.data_ptr()),
                                          C.c_void_p(s.cuda_stream))

    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert call() == 0, L.st_last_error()
    torch.cuda.synchronize()
    r0, n0 = r.clone(), norm.clone()
    r_ref = f.cpu().numpy() - O.assemble(om, g) @ x.cpu().numpy()
    assert rel_err(r0.cpu().numpy(), r_ref) < 1e-12
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        code = call()
    assert code == 0, L.st_last_error()
    for _ in range(2):
        r.fill_(float("nan"))
        norm.fill_(float("nan"))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(r, r0) and torch.equal(norm, n0)


def test_residual_norm_noalloc_rejects_planes_beyond_its_scratch():
    L = ensure_built()
    from paper_2508_09589_gb300 import mesh_desc
    d = mesh_desc((2048, 2048), 2)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    code = L.st_residual_norm_noalloc(C.byref(d), p, 0, p, p, p, p, None)
    assert code == -1
    assert b"scratch" in L.st_last_error()
