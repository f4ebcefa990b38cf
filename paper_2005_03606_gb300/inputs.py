"""Seeded synthetic inputs: material fields eps(x) and problem workloads.

This module only draws parameters (mode wavenumbers, phases, box corners,
noise vectors) from a seed; it holds none of the method's arithmetic.  Both
the CUDA library and the CPU oracle receive the drawn parameters as plain
numbers and evaluate eps(x) with their own code.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here so that the
same seed gives the same field on every machine and numpy version.

Field families (the paper's workloads are analytic eps fields, Section
"Results"; the families below stand in for them and for the lognormal/box
fields of the benchmark workloads):

* ``const``   eps = v_out everywhere (the "constant eps" case of Section
  "Numerical computation of stencils").
* ``disc``    eps = v_in where |x - c| < r, else v_out.
* ``fourier`` eps = v_out * exp(sigma*sqrt(2/M) * sum_m cos(2 pi k_m.x + phi_m)),
  optionally times ``jump_factor`` where x_0 >= jump_x.  k_m are integer
  vectors with components in [-kmax, kmax] and 1 <= max|k_m| <= kmax.
* ``boxes``   eps = v_in inside the union of axis-aligned boxes
  [lo, hi) (half-open), else v_out.
* ``theta``   eps = 1 + (0.3/d) prod_i exp(-theta x_i) cos(pi theta x_i)
  (the paper's first test setup, Eq. "theta-setup").
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

MAX_MODES = 32
MAX_BOXES = 64

KIND_CONST, KIND_DISC, KIND_FOURIER, KIND_BOXES, KIND_THETA = 0, 1, 2, 3, 4
KIND_NAMES = {"const": KIND_CONST, "disc": KIND_DISC, "fourier": KIND_FOURIER,
              "boxes": KIND_BOXES, "theta": KIND_THETA}

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based 64-bit generator (splitmix64)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive), by rejection-free modulo (tiny bias is irrelevant here)."""
        return lo + self.next_u64() % (hi - lo + 1)


@dataclasses.dataclass
class EpsField:
    """Parameters of one material field; all values are plain numbers."""

    kind: int
    dim: int
    v_out: float = 1.0
    v_in: float = 1.0
    center: Sequence[float] = (0.5, 0.5, 0.5)
    radius: float = 0.0
    sigma: float = 0.0
    theta: float = 0.0
    jump_x: float = 2.0          # outside [0,1]: no jump
    jump_factor: float = 1.0
    k: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.int32))
    phase: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    box_lo: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3)))
    box_hi: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3)))

    @property
    def n_modes(self) -> int:
        return int(self.k.shape[0])

    @property
    def n_boxes(self) -> int:
        return int(self.box_lo.shape[0])


def const_field(dim: int, value: float = 1.0) -> EpsField:
    return EpsField(KIND_CONST, dim, v_out=float(value))


def disc_field(dim: int, v_in: float = 10.0, v_out: float = 1.0,
               center=(0.5, 0.5, 0.5), radius: float = 0.3) -> EpsField:
    return EpsField(KIND_DISC, dim, v_out=float(v_out), v_in=float(v_in),
                    center=tuple(float(c) for c in center), radius=float(radius))


def theta_field(dim: int, theta: float) -> EpsField:
    return EpsField(KIND_THETA, dim, theta=float(theta))


def fourier_field(dim: int, seed: int, sigma: float = 1.0, n_modes: int = 16,
                  kmax: int = 8, base: float = 1.0, jump_x: Optional[float] = None,
                  jump_factor: float = 1.0) -> EpsField:
    """Lognormal field from ``n_modes`` random Fourier modes (wavenumbers 1..kmax)."""
    if not 1 <= n_modes <= MAX_MODES:
        raise ValueError("n_modes out of range")
    rng = SplitMix64(seed)
    k = np.zeros((n_modes, 3), np.int32)
    phase = np.zeros(n_modes)
    for m in range(n_modes):
        while True:
            kv = [rng.randint(-kmax, kmax) for _ in range(dim)]
            if max(abs(v) for v in kv) >= 1:
                break
        k[m, :dim] = kv
        phase[m] = rng.uniform(0.0, 2.0 * math.pi)
    return EpsField(KIND_FOURIER, dim, v_out=float(base), sigma=float(sigma), k=k,
                    phase=phase, jump_x=2.0 if jump_x is None else float(jump_x),
                    jump_factor=float(jump_factor))


def boxes_field(dim: int, seed: int, n_boxes: int = 64, contrast: float = 1e3,
                side=(0.02, 0.15), background: float = 1.0) -> EpsField:
    """Union of ``n_boxes`` axis-aligned boxes with eps = contrast*background inside."""
    if not 1 <= n_boxes <= MAX_BOXES:
        raise ValueError("n_boxes out of range")
    rng = SplitMix64(seed)
    lo = np.zeros((n_boxes, 3))
    hi = np.zeros((n_boxes, 3))
    for b in range(n_boxes):
        for a in range(dim):
            w = rng.uniform(side[0], side[1])
            l0 = rng.uniform(0.0, 1.0 - w)
            lo[b, a], hi[b, a] = l0, l0 + w
    return EpsField(KIND_BOXES, dim, v_out=float(background),
                    v_in=float(background * contrast), box_lo=lo, box_hi=hi)


def noise_vector(dim: int, n_cells: int, seed: int, lo: float = 0.0,
                 hi: float = 4.0 / 3.0) -> np.ndarray:
    """Seeded noise on the (n+1)^d vertex grid, zero on the Dirichlet boundary.

    The paper initialises its runs with noise from [0, 4/3] (Section "Results").
    """
    n1 = n_cells + 1
    rng = SplitMix64(seed)
    u = np.array([rng.uniform(lo, hi) for _ in range(n1 ** dim)], dtype=np.float64)
    u = u.reshape((n1,) * dim)
    sl = [slice(None)] * dim
    for a in range(dim):
        for edge in (0, n1 - 1):
            s2 = list(sl)
            s2[a] = edge
            u[tuple(s2)] = 0.0
    return u.reshape(-1)


@dataclasses.dataclass
class Workload:
    """A problem instance: -div(eps grad u) = f_const on [0,1]^d, u = 0 on the boundary."""

    name: str
    dim: int
    n_cells: int
    eps: EpsField
    s_final: int
    s_schedule: List[int]
    f_const: float = 1.0


def _check_pow3(n: int) -> None:
    m = n
    while m % 3 == 0 and m > 1:
        m //= 3
    if m != 1 or n < 3:
        raise ValueError(f"n_cells={n} is not a power of 3")


def workload(name: str, n_cells: Optional[int] = None) -> Workload:
    """The benchmark workloads, optionally at a smaller ``n_cells`` for tests."""
    if name == "disc2d":          # 2D 81^2, eps = 10 inside r=0.3, s = 8
        n = n_cells or 81
        w = Workload(name, 2, n, disc_field(2), 8, [8])
    elif name == "fourier3d":     # 3D 81^3 lognormal sigma=1, 16 modes, s = 1->2->4->8
        n = n_cells or 81
        w = Workload(name, 3, n, fourier_field(3, 2002, sigma=1.0), 8, [1, 2, 4, 8])
    elif name == "boxes3d":       # 3D 243^3, 64 boxes contrast 1e3, s to 8
        n = n_cells or 243
        w = Workload(name, 3, n, boxes_field(3, 2003), 8, [1, 2, 4, 8])
    elif name == "jump3d":        # 3D 243^3 lognormal sigma=2 x 1e4 for x >= 0.37, s to 16
        n = n_cells or 243
        w = Workload(name, 3, n, fourier_field(3, 2005, sigma=2.0, jump_x=0.37,
                                                jump_factor=1e4), 16, [1, 2, 4, 8, 16])
    else:
        raise KeyError(name)
    _check_pow3(w.n_cells)
    return w


SERVING_SIZES = [(3, 27), (3, 81), (3, 243), (2, 243), (2, 729)]


def serving_requests(n_requests: int = 512, seed: int = 2004, rate_per_s: float = 1.0,
                     sizes=SERVING_SIZES) -> List[dict]:
    """Seeded request stream: size uniform over ``sizes``, lognormal eps with
    sigma ~ U[0.5, 2], Poisson arrivals (exponential gaps) at ``rate_per_s``."""
    rng = SplitMix64(seed)
    out = []
    t = 0.0
    for i in range(n_requests):
        dim, n = sizes[rng.randint(0, len(sizes) - 1)]
        sigma = rng.uniform(0.5, 2.0)
        fseed = rng.next_u64() & 0xFFFFFFFF
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        out.append({"id": i, "dim": dim, "n_cells": n, "sigma": sigma,
                    "eps": fourier_field(dim, fseed, sigma=sigma), "arrival_s": t})
    return out
