"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the bench.

This module holds input data only: mesh sizes, material constants, boundary
condition kinds, source kinds and seeded random design fields.  It contains
none of the discretisation or solver arithmetic, so both sides of every parity
test can use it without sharing any of the method.

Design fields follow the recipe used for every random workload: white
standard-normal noise on the element grid (numpy PCG64, fixed seed), smoothed
by a periodic Gaussian kernel through the FFT, normalised to zero mean and unit
standard deviation, and mapped to [0, 1] by the logistic function.  The
logistic map and the FFT smoothing are properties of the input distribution,
not of the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

# Paper defaults (Sec. 2.2, after the SIMP equations): C_ins, C_con, k_ins, k_con, p_c, p_k.
PAPER_MATERIAL = dict(C_ins=0.5, C_con=1.0, k_ins=0.03, k_con=3.0, p_c=2, p_k=3)
# Workload material "k_min/k_max = 1e-3, unit heat capacity": C identical for both phases.
UNIT_CAPACITY_MATERIAL = dict(C_ins=1.0, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)
# 3+1D workload: capacity varied independently of conductivity (SIMP p=1 over [0.5, 1]).
CAPACITY_VARIED_MATERIAL = dict(C_ins=0.5, C_con=1.0, k_ins=1e-3, k_con=1.0, p_c=1, p_k=3)


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: mesh, material, boundary condition, source, design."""
    name: str
    ns: Tuple[int, ...]          # spatial element counts (x first)
    nt: int                      # time element count
    material: dict
    bc: str = "patch_left"       # patch_left | patch_bottom | all_walls | none
    bc_width: float = 0.1        # patch width as a fraction of the edge length
    tau: float = 1.0
    source: str = "uniform"      # uniform | sin_t
    source_q0: float = 1.0
    source_a: float = 1.0        # sin_t: q(t) = q0 * (a + b sin(2 pi f t))
    source_b: float = 0.5
    source_f: float = 4.0
    design: str = "uniform"      # uniform | grf_extruded | grf_spacetime
    design_value: float = 0.5
    corr_len: float = 0.05       # correlation length in domain units (std of the kernel)
    seed: int = 1

    @property
    def sd(self) -> int:
        return len(self.ns)

    @property
    def n_dofs(self) -> int:
        n = self.nt + 1
        for k in self.ns:
            n *= k + 1
        return n

    @property
    def n_elem(self) -> int:
        n = self.nt
        for k in self.ns:
            n *= k
        return n

    @property
    def extruded(self) -> bool:
        return self.design in ("uniform", "grf_extruded")

    def design_shape(self) -> Tuple[int, ...]:
        """Design array shape, C order with x fastest: ([nt,] [nz,] ny, nx)."""
        sp = tuple(reversed(self.ns))
        return sp if self.extruded else (self.nt,) + sp


def grf_sigmoid(shape: Tuple[int, ...], sigma_cells: Tuple[float, ...], seed: int) -> np.ndarray:
    """Seeded smooth random field in (0, 1).

    shape and sigma_cells are in the same (C-order) axis order.  The kernel is a
    periodic Gaussian with standard deviation sigma_cells[d] cells on axis d.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(shape)
    zf = np.fft.fftn(z)
    for d, (n, s) in enumerate(zip(shape, sigma_cells)):
        k = np.fft.fftfreq(n)  # cycles per cell
        g = np.exp(-2.0 * (math.pi * s * k) ** 2)  # FT of a unit-mass Gaussian
        bshape = [1] * len(shape)
        bshape[d] = n
        zf = zf * g.reshape(bshape)
    z = np.real(np.fft.ifftn(zf))
    z = (z - z.mean()) / z.std()
    return 1.0 / (1.0 + np.exp(-z))


def make_design(w: Workload) -> np.ndarray:
    """The design array of a workload (float64, C order, x fastest)."""
    shape = w.design_shape()
    if w.design == "uniform":
        return np.full(shape, w.design_value, dtype=np.float64)
    if w.design == "grf_extruded":
        sig = tuple(w.corr_len * n for n in reversed(w.ns))
        return grf_sigmoid(shape, sig, w.seed)
    if w.design == "grf_spacetime":
        sig = (w.corr_len * w.nt / w.tau,) + tuple(w.corr_len * n for n in reversed(w.ns))
        return grf_sigmoid(shape, sig, w.seed)
    raise ValueError(w.design)


# The five workloads: sizes, materials, boundary conditions, sources and designs.
C0 = Workload("c0_32x32x32_fp64", (32, 32), 32, UNIT_CAPACITY_MATERIAL,
              design="uniform", design_value=0.5)
C1 = Workload("c1_256x256x256_grf_extruded", (256, 256), 256, UNIT_CAPACITY_MATERIAL,
              design="grf_extruded", seed=1)
C2 = Workload("c2_512x512x256_grf_spacetime_sin", (512, 512), 256, UNIT_CAPACITY_MATERIAL,
              design="grf_spacetime", source="sin_t", seed=2)
C3 = Workload("c3_64x64x64x64_grf_extruded_3d", (64, 64, 64), 64, CAPACITY_VARIED_MATERIAL,
              design="grf_extruded", seed=4)

WORKLOADS = {w.name: w for w in (C0, C1, C2, C3)}


def scaled(w: Workload, ns: Tuple[int, ...], nt: int, name: Optional[str] = None) -> Workload:
    """Same family (material, bc, source, design recipe) at another mesh size."""
    return replace(w, ns=tuple(ns), nt=nt, name=name or f"{w.name}@{'x'.join(map(str, ns))}x{nt}")


def serving_requests(n: int = 256, seed: int = 7, lo: int = 32, hi: int = 512,
                     t_lo: int = 32, t_hi: int = 256, multiple: int = 16):
    """Serving stream: per-axis counts log-uniform in [lo, hi] (time [t_lo, t_hi]),
    rounded to a multiple of 16; each request has its own seeded extruded design."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(n):
        def draw(a, b):
            v = math.exp(rng.uniform(math.log(a), math.log(b)))
            return int(max(multiple, round(v / multiple) * multiple))
        nx, ny, nt = draw(lo, hi), draw(lo, hi), draw(t_lo, t_hi)
        out.append(Workload(f"req{r}_{nx}x{ny}x{nt}", (nx, ny), nt, UNIT_CAPACITY_MATERIAL,
                            design="grf_extruded", seed=1000 + r))
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 11) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
