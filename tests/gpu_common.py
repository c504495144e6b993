"""Shared helpers of the GPU tests: building the native library, seeded cases, BF16 rounding."""
import math
import os

import numpy as np

from oracle import st_oracle as O


def ensure_built():
    from paper_2508_09589_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2508_09589_gb300 import build
        build.build()
    return _lib.lib()


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest BF16 value (ties to even), exactly in float64:
    x = m 2^e with m in [0.5, 1); BF16 keeps 8 significant bits."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def mat_dict(mat: O.Material) -> dict:
    return dict(C_ins=mat.C_ins, C_con=mat.C_con, k_ins=mat.k_ins, k_con=mat.k_con, p_c=mat.p_c, p_k=mat.p_k)


def gpu_mesh(om: O.Mesh, **kw):
    from paper_2508_09589_gb300 import Mesh
    return Mesh(om.ns, om.nt, ext=om.ext, tau=om.tau, material=mat_dict(om.mat), bc=om.bc,
                bc_width=om.bc_width, **kw)


def oracle_levels(om: O.Mesh, gm_levels):
    """Oracle Level objects matching the hierarchy the library built."""
    out = []
    for L in gm_levels:
        h = tuple(e / n for e, n in zip(om.ext, L["ns"]))
        out.append(O.Level(tuple(L["ns"]), L["nt"], h, om.tau / L["nt"], L["to_next"]))
    return out


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def parity_rtol(A, s, f) -> float:
    """Outer tolerance for tight parity runs: 1e-13, raised to 20x the FP64 residual floor
    || |A| |s| || u / ||f|| when the problem's scaling puts the floor above it (the exact
    solution's own residual in FP64 arithmetic is about that floor)."""
    floor = np.linalg.norm(abs(A) @ np.abs(s)) * 1.11e-16 / np.linalg.norm(f)
    return max(1e-13, 20.0 * floor)


U32 = 2.0 ** -24
U64 = 2.0 ** -53


def rowwise_excess(y, yref, B, x, c, u) -> float:
    """Largest ratio |y - yref|_i / (c u (B |x|)_i) over the rows: the componentwise rounding
    bound of an evaluation that sums terms bounded by B |x| (B the element-wise absolute
    operator or a product of non-negative transfers).  <= 1 means every row is within it."""
    y = np.asarray(y, dtype=np.float64)
    yref = np.asarray(yref, dtype=np.float64)
    allowed = c * u * (B @ np.abs(np.asarray(x, dtype=np.float64))) + 1e-300
    return float((np.abs(y - yref) / allowed).max())


def galerkin_abs(B, Pt, cmask):
    """Bound matrix of the next coarser level: Pt^T B Pt with the identity on prescribed nodes.
    The element blocks of the Galerkin operator satisfy |P_E^T (sum_e J_e) P_E| <= P_E^T (sum_e
    |J_e|) P_E because P >= 0, so this bounds their entry-wise absolute sum."""
    import scipy.sparse as sp
    return (Pt.T @ B @ Pt + sp.diags(cmask.astype(np.float64))).tocsr()
