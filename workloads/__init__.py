"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws numbers: it holds none of the force or integrator
arithmetic. Every generator returns plain NumPy arrays in physical units
(FP64 as drawn, plus the FP32-rounded copy that both the CUDA path and the
oracle consume, so that the two see bit-identical inputs).

Workloads (the paper's own runs used no public dataset for gravity, and its
molecular-dynamics protein, lambda repressor with 1280 atoms, is not
available; the random atom sphere below stands in for it):

* :func:`plummer`       -- Plummer sphere, G = M = a = 1, m = 1/N, sampled
  with the Aarseth-Henon-Wielen (1974) method, centre of mass at rest.
* :func:`ljc_sphere`    -- N atoms uniform in a sphere, >= 1 A apart,
  4 atom types with sigma in [2.5, 3.8] A and epsilon in [0.05, 0.2]
  kcal/mol, charges uniform in [-0.8, 0.8] e shifted to total 0.
* :func:`ensemble`      -- many independent systems with N log-uniform in
  [64, 4096], alternating Plummer gravity and LJ + Coulomb spheres.
* :func:`perturbed_target` -- x* = x + 0.01 xi, xi ~ N(0, I).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ATOM_MASSES = np.array([12.011, 14.007, 15.999, 32.06])  # amu, per type (C, N, O, S)


def plummer_softening(n: int) -> float:
    """Softening of the large gravity workload: eps = 0.04 * N^(-1/3)."""
    return 4.0 / n ** (1.0 / 3.0) * 0.01


@dataclass
class GravInput:
    x: np.ndarray          # (n, 3) float64 positions as drawn
    v: np.ndarray          # (n, 3) float64 velocities
    m: np.ndarray          # (n,)   float64 masses
    eps: float = 0.01
    G: float = 1.0
    seed: int = 0

    @property
    def n(self) -> int:
        return self.x.shape[0]

    def f32(self):
        """FP32-rounded (x, v, m) -- the values both paths consume."""
        return (self.x.astype(np.float32), self.v.astype(np.float32),
                self.m.astype(np.float32))

    def f32_as_f64(self):
        x, v, m = self.f32()
        return x.astype(np.float64), v.astype(np.float64), m.astype(np.float64)


@dataclass
class LJCInput:
    x: np.ndarray          # (n, 3) positions, Angstrom
    v: np.ndarray          # (n, 3) velocities (zero)
    m: np.ndarray          # (n,) masses, amu
    q: np.ndarray          # (n,) partial charges, e (sum exactly 0 in FP64)
    types: np.ndarray      # (n,) int32 atom types
    sig_t: np.ndarray      # (ntypes,) sigma per type, Angstrom
    eps_t: np.ndarray      # (ntypes,) epsilon per type, kcal/mol
    dielectric: float = 80.0
    seed: int = 2

    @property
    def n(self) -> int:
        return self.x.shape[0]

    def f32(self):
        """FP32-rounded (x, v, m, q, sig_t, eps_t)."""
        f = np.float32
        return (self.x.astype(f), self.v.astype(f), self.m.astype(f), self.q.astype(f),
                self.sig_t.astype(f), self.eps_t.astype(f))

    def f32_as_f64(self):
        return tuple(a.astype(np.float64) for a in self.f32())


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def plummer(n: int, seed: int = 0, eps: float | None = None, mass_cut: float = 0.999,
            rng: np.random.Generator | None = None) -> GravInput:
    """Plummer sphere (a = G = M = 1), Aarseth, Henon & Wielen (1974).

    Radius from the cumulative mass X ~ U(0, mass_cut]: r = (X^(-2/3) - 1)^(-1/2).
    Speed v = q * sqrt(2) * (1 + r^2)^(-1/4) with q drawn by von Neumann
    rejection from g(q) = q^2 (1 - q^2)^(7/2) (maximum < 0.1). Directions are
    isotropic; the centre of mass is moved to rest at the origin.
    """
    rng = rng if rng is not None else np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.0, 1.0, n) * mass_cut
    X = np.where(X <= 0.0, mass_cut * 1e-12, X)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _unit_vectors(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.uniform(0.0, 1.0, todo.size)
        x5 = rng.uniform(0.0, 1.0, todo.size)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = speed[:, None] * _unit_vectors(rng, n)
    m = np.full(n, 1.0 / n)
    x -= np.sum(m[:, None] * x, axis=0) / m.sum()
    v -= np.sum(m[:, None] * v, axis=0) / m.sum()
    return GravInput(x=x, v=v, m=m, eps=0.01 if eps is None else float(eps), seed=seed)


def _place_in_sphere(rng: np.random.Generator, n: int, radius: float, min_sep: float):
    """Uniform points in a ball, rejecting any within ``min_sep`` of another."""
    cell = min_sep
    grid: dict[tuple[int, int, int], list[int]] = {}
    pts = np.empty((n, 3))
    k = 0
    r2min = min_sep * min_sep
    while k < n:
        batch = rng.uniform(-radius, radius, (4096, 3))
        batch = batch[np.einsum("ij,ij->i", batch, batch) <= radius * radius]
        for p in batch:
            c = tuple(int(math.floor(p[a] / cell)) for a in range(3))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for idx in grid.get((c[0] + dx, c[1] + dy, c[2] + dz), ()):
                            d = pts[idx] - p
                            if d @ d < r2min:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pts[k] = p
                grid.setdefault(c, []).append(k)
                k += 1
                if k == n:
                    break
    return pts


def ljc_sphere(n: int = 8192, seed: int = 2, radius: float | None = None,
               min_sep: float = 1.0, ntypes: int = 4, dielectric: float = 80.0,
               rng: np.random.Generator | None = None,
               type_params: tuple[np.ndarray, np.ndarray] | None = None) -> LJCInput:
    """Random atoms in a sphere for the LJ + Coulomb (continuum solvent) law.

    Radius 45 A for 8192 atoms; other sizes keep that density
    (R = 45 (N / 8192)^(1/3)). Types uniform over 4; sigma_t ~ U[2.5, 3.8] A,
    epsilon_t ~ U[0.05, 0.2] kcal/mol; charges ~ U[-0.8, 0.8] e minus their
    mean so the total is 0; masses per type {C, N, O, S}; velocities 0.
    """
    rng = rng if rng is not None else np.random.Generator(np.random.PCG64(seed))
    if radius is None:
        radius = 45.0 * (n / 8192.0) ** (1.0 / 3.0)
    if type_params is None:
        sig_t = rng.uniform(2.5, 3.8, ntypes)
        eps_t = rng.uniform(0.05, 0.2, ntypes)
    else:
        sig_t, eps_t = (np.asarray(a, dtype=np.float64) for a in type_params)
    x = _place_in_sphere(rng, n, radius, min_sep)
    types = rng.integers(0, ntypes, n).astype(np.int32)
    q = rng.uniform(-0.8, 0.8, n)
    q = q - q.mean()
    m = ATOM_MASSES[types % len(ATOM_MASSES)].astype(np.float64)
    v = np.zeros((n, 3))
    return LJCInput(x=x, v=v, m=m, q=q, types=types, sig_t=sig_t, eps_t=eps_t,
                    dielectric=dielectric, seed=seed)


@dataclass
class Ensemble:
    systems: list = field(default_factory=list)   # GravInput | LJCInput, in order
    sig_t: np.ndarray | None = None
    eps_t: np.ndarray | None = None

    @property
    def sizes(self) -> np.ndarray:
        return np.array([s.n for s in self.systems], dtype=np.int64)


def ensemble(nsys: int = 512, seed: int = 3, nmin: int = 64, nmax: int = 4096) -> Ensemble:
    """Independent systems, N log-uniform in [nmin, nmax], even index gravity
    (Plummer, eps = 0.01), odd index LJ + Coulomb at the 8192-atom density.
    All LJ systems share one table of 4 atom types."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nsys))
    sizes = np.clip(np.rint(sizes).astype(np.int64), nmin, nmax)
    sig_t = rng.uniform(2.5, 3.8, 4)
    eps_t = rng.uniform(0.05, 0.2, 4)
    out = Ensemble(sig_t=sig_t, eps_t=eps_t)
    for k, n in enumerate(sizes):
        sub = np.random.Generator(np.random.PCG64([seed, k]))
        if k % 2 == 0:
            out.systems.append(plummer(int(n), eps=0.01, rng=sub))
        else:
            out.systems.append(ljc_sphere(int(n), rng=sub, type_params=(sig_t, eps_t)))
    return out


def perturbed_target(x: np.ndarray, seed: int = 4, scale: float = 0.01) -> np.ndarray:
    """x* = x + scale * xi with xi ~ N(0, I) (the adjoint workload's target)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asarray(x, dtype=np.float64) + scale * rng.standard_normal(np.shape(x))


def random_directions(shape, k: int, seed: int = 5) -> np.ndarray:
    """k unit directions in R^shape for directional finite differences."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((k,) + tuple(shape))
    d /= np.sqrt(np.sum(d.reshape(k, -1) ** 2, axis=1)).reshape((k,) + (1,) * len(shape))
    return d
