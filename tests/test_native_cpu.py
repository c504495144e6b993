"""CPU-side checks of the native library: it loads, exports every symbol include/st.h
declares, and its host-only logic (Algorithm 1 planner, footprint model, argument
validation) behaves.  No kernel runs here."""
import os
import re

import numpy as np
import pytest

from oracle import st_oracle as O
from tests.gpu_common import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    return ensure_built()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "st.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][^\n;()]*?\b(st_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(L):
    names = _declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n
    from paper_2508_09589_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)
    assert L.st_version().startswith(b"st-gb300")


def _golden():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "paper_hierarchies.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            case, tau, matl, levels = [p.strip() for p in line.split("|")]
            Ci, Cc, ki, kc = map(float, matl.split())
            rows.append((case, float(tau), dict(C_ins=Ci, C_con=Cc, k_ins=ki, k_con=kc),
                         [tuple(map(int, x.split("x"))) for x in levels.split()]))
    return rows


@pytest.mark.parametrize("case,tau,mat,levels", _golden())
def test_native_algorithm1_reproduces_paper_tables(L, case, tau, mat, levels):
    from paper_2508_09589_gb300 import plan_hierarchy
    got = plan_hierarchy((640, 640), 1280, tau=tau, material=mat, max_levels=len(levels), coarse_dof_cap=1)
    assert [(g["ns"][0], g["ns"][1], g["nt"]) for g in got] == levels


@pytest.mark.parametrize("ns,nt,mat,cap", [
    ((256, 256), 256, dict(C_ins=1, C_con=1, k_ins=1e-3, k_con=1, p_c=1, p_k=3), 2000),
    ((512, 512), 256, dict(C_ins=1, C_con=1, k_ins=1e-3, k_con=1, p_c=1, p_k=3), 2000),
    ((64, 64, 64), 64, dict(C_ins=0.5, C_con=1, k_ins=1e-3, k_con=1, p_c=1, p_k=3), 2000),
    ((36, 20), 16, dict(C_ins=1, C_con=1, k_ins=1e-3, k_con=1, p_c=1, p_k=3), 300),
    ((96, 48), 160, dict(), 1000),
])
def test_native_planner_matches_oracle_hierarchy(L, ns, nt, mat, cap):
    from paper_2508_09589_gb300 import plan_hierarchy
    got = plan_hierarchy(ns, nt, material=mat, coarse_dof_cap=cap)
    om = O.Mesh(ns, nt, mat=O.Material(**{**dict(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3), **mat}))
    ref = O.hierarchy(om, coarse_cap=cap)
    assert [(g["ns"], g["nt"], g["to_next"]) for g in got] == [(tuple(r.ns), r.nt, r.to_next) for r in ref]


def test_workload_hierarchies():
    """Hierarchies of the 256^2 x 256 workload under the k ratio 1e-3 / unit capacity."""
    from paper_2508_09589_gb300 import plan_hierarchy
    got = plan_hierarchy((256, 256), 256, material=dict(C_ins=1, C_con=1, k_ins=1e-3, k_con=1, p_c=1, p_k=3))
    assert [g["ns"][0] for g in got] == [256, 128, 64, 32, 32, 32, 16, 16, 16, 8]
    assert [g["nt"] for g in got] == [256, 256, 256, 256, 128, 64, 64, 32, 16, 16]


def test_footprint_model_and_argument_validation(L):
    from paper_2508_09589_gb300 import footprint_bytes, plan_hierarchy, STError
    a = footprint_bytes((64, 64), 64)
    b = footprint_bytes((128, 128), 64)
    c = footprint_bytes((64, 64), 64, precision="fp64")
    assert 0 < a < b and a < c
    # a Jacobi-smoothed hierarchy keeps no Krylov basis on its levels
    j = footprint_bytes((64, 64), 64, smoother="jacobi")
    assert 0 < j < a
    with pytest.raises(STError):
        plan_hierarchy((64, 64), 0)
    with pytest.raises(STError):
        plan_hierarchy((64, 64), 8, material=dict(p_k=0))


def test_create_mesh_without_gpu_fails_cleanly(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2508_09589_gb300 import Mesh, STError
    with pytest.raises(STError) as e:
        Mesh((8, 8), 8)
    assert e.value.code == -6


@pytest.mark.parametrize("ns,nt,cap", [((32, 32), 32, 300), ((64, 48), 16, 500), ((16, 16, 16), 16, 300)])
def test_full_coarsening_planner_matches_oracle(L, ns, nt, cap):
    """Full space-time coarsening (the ablation of Sec. 5.1.2): every level halves space and time
    together while both can be halved, as the oracle's hierarchy in mode 'full'."""
    from paper_2508_09589_gb300 import plan_hierarchy
    om = O.Mesh(ns, nt, mat=O.Material(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3))
    ref = O.hierarchy(om, coarse_cap=cap, mode="full")
    got = plan_hierarchy(ns, nt, material=dict(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3),
                         coarse_dof_cap=cap, coarsening="full")
    assert [(tuple(L_.ns), L_.nt, L_.to_next) for L_ in ref] == [(g["ns"], g["nt"], g["to_next"]) for g in got]
    assert all(g["to_next"] in ("full", "") for g in got)


def test_optimiser_loop_and_reference_argument_checks_without_a_gpu(L):
    """Host-side argument checks of the MMA, the design loop, the BDF1 reference and the smoother
    option, each refused before any device work."""
    import ctypes as C
    from paper_2508_09589_gb300 import _lib as LB, mesh_desc, plan_hierarchy, STError
    h = C.c_void_p()
    assert L.st_mma_create(0, None, C.byref(h)) == -1
    for field, bad in (("decr", 1.5), ("lam_max", float("inf")), ("move", float("nan")), ("s0", 0.0)):
        p = LB.MmaParams()
        L.st_mma_params_default(C.byref(p))
        setattr(p, field, bad)
        assert L.st_mma_create(10, C.byref(p), C.byref(h)) == -1, field
    g = np.full(16, 0.5)
    assert L.st_topopt_create(None, None, C.c_void_p(g.ctypes.data), 0, 16, 0, C.byref(h)) == -1
    d = mesh_desc((8, 8), 0)
    assert L.st_bdf1_create(C.byref(d), C.byref(h)) == -1
    with pytest.raises(STError):
        plan_hierarchy((64, 64), 8, smoother="jacobi", smoother_omega=1.5)
    assert len(plan_hierarchy((64, 64), 8, smoother="jacobi", smoother_omega=0.5)) >= 2
