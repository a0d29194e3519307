"""FP64 CPU oracle for the all-pairs N-body method of arXiv 0706.3060.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library never links, imports or calls anything here, and
nothing here imports the CUDA library.

What it computes (each item is the plain definition, no blocking or fusion):

* :func:`grav_accel`     -- Eq. 1 (Sec. 3.3), Table 1 "Gravity (accel)":
  a_i = -G sum_{j!=i} m_j r_ij / (r_ij^2 + eps^2)^{3/2}, plus the potential.
* :func:`grav_jerk`      -- Table 1 "Gravity (accel & jerk)": acceleration and
  its time derivative (jerk) for a 4th-order Hermite scheme.
* :func:`ljc_force`      -- Table 1 "LJC(constant)", read as the standard
  12-6 Lennard-Jones force plus Coulomb in a dielectric eps_r, with
  Lorentz-Berthelot mixing (the paper prints the LJ term without its 24/r^2
  factor; see ``nbody_oracle.c``).
* :func:`leapfrog`       -- kick-drift-kick leapfrog, the update step of
  Sec. 1 (the paper leaves the integrator open; KDK is the reading used).
* :func:`grav_vjp`, :func:`ljc_vjp` -- J^T lambda of the force laws above,
  block by block from the Jacobian, with mass and per-type sigma/epsilon
  derivatives.
* :func:`adjoint_leapfrog` -- reverse-mode KDK with every state stored.
* :func:`hermite`        -- fourth-order Hermite steps on acceleration + jerk.
* :func:`diagnostics`    -- kinetic and potential energy, momentum and
  angular momentum in FP64.

Pins (``tests/test_oracle_*.py``) tie each function to something other than
itself: closed forms (two-body force, Kepler orbit, LJ minimum, Plummer
potential energy), high-precision brute force, Newton's third law,
F = -grad U by finite differences, invariances, and finite differences of the
loss for the adjoint.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

COULOMB_K = 332.0637  # kcal * A / (mol * e^2), reading C2 (units A, kcal/mol, e)


def build(force: bool = False) -> str:
    """Compile ``nbody_oracle.c`` into ``liboracle.so`` with the host gcc."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64 = ctypes.c_int64
            lib.oracle_grav.argtypes = [i64, d, d, ctypes.c_double, ctypes.c_double,
                                        i64, i64p, d, d]
            lib.oracle_ljc.argtypes = [i64, d, d, d, d, ctypes.c_double, i64, i64p, d, d]
            lib.oracle_grav_jerk.argtypes = [i64, d, d, d, ctypes.c_double, ctypes.c_double,
                                             i64, i64p, d, d]
            lib.oracle_grav_jerk.restype = None
            lib.oracle_ljc_model.argtypes = [i64, d, d, d, d, ctypes.c_double, ctypes.c_int,
                                             i64, i64p, d, d]
            lib.oracle_ljc_model.restype = None
            lib.oracle_grav_vjp.argtypes = [i64, d, d, ctypes.c_double, ctypes.c_double,
                                            d, d, d]
            lib.oracle_grav_vjp_rows.argtypes = [i64, d, d, ctypes.c_double, ctypes.c_double,
                                                 d, i64, i64p, d, d]
            lib.oracle_grav_vjp_rows.restype = None
            lib.oracle_ljc_vjp.argtypes = [i64, d, d, d, i32p, ctypes.c_int32, d, d,
                                           ctypes.c_double, d, d, d, d, d]
            lib.oracle_ljc_vjp_model.argtypes = [i64, d, d, d, i32p, ctypes.c_int32, d, d,
                                                 ctypes.c_double, ctypes.c_int, d, d, d, d, d]
            lib.oracle_ljc_vjp_model.restype = None
            lib.oracle_threads.argtypes = [ctypes.c_int]
            lib.oracle_threads.restype = ctypes.c_int
            for f in (lib.oracle_grav, lib.oracle_ljc, lib.oracle_grav_vjp,
                      lib.oracle_ljc_vjp):
                f.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _idx(idx):
    if idx is None:
        return None, None
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    return idx, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def set_threads(n: int | None) -> int:
    """Set the OpenMP thread count of the compiled oracle (None: leave it);
    returns the count in force."""
    return int(_load().oracle_threads(0 if n is None else int(n)))


# ---------------------------------------------------------------------------
# Force laws
# ---------------------------------------------------------------------------
def grav_accel(x, m, G=1.0, eps=0.0, idx=None, potential=False):
    """Eq. 1: softened gravitational acceleration on particles ``idx``.

    x: (n, 3), m: (n,). Returns acc (ni, 3) and, if ``potential``, phi (ni,)
    with phi_i = -G sum_{j!=i} m_j / sqrt(r^2 + eps^2).
    """
    lib = _load()
    x = _f64(x, (-1, 3))
    m = _f64(m)
    n = x.shape[0]
    idx, idxp = _idx(idx)
    ni = n if idx is None else idx.shape[0]
    acc = np.zeros((ni, 3))
    phi = np.zeros(ni) if potential else None
    lib.oracle_grav(n, _dp(x), _dp(m), float(G), float(eps) ** 2, ni, idxp, _dp(acc),
                    _dp(phi))
    return (acc, phi) if potential else acc


def grav_jerk(x, v, m, G=1.0, eps=0.0, idx=None):
    """Table 1 "Gravity (accel & jerk)": returns (acc (ni,3), jerk (ni,3)) on the
    targets ``idx`` (all particles if None), the jerk being the time derivative of
    the acceleration for particles moving at v."""
    lib = _load()
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    m = _f64(m)
    n = x.shape[0]
    idx, ip = _idx(idx)
    ni = n if idx is None else idx.shape[0]
    acc = np.zeros((ni, 3))
    jerk = np.zeros((ni, 3))
    lib.oracle_grav_jerk(n, _dp(x), _dp(v), _dp(m), float(G), float(eps) ** 2, ni, ip,
                         _dp(acc), _dp(jerk))
    return acc, jerk


def ljc_force(x, q, sig, eps, kq=COULOMB_K / 80.0, idx=None, potential=False, linear=False):
    """Table 1 LJC(constant): Coulomb with dielectric plus 12-6 Lennard-Jones.

    Per-particle q, sig, eps (n,); ``kq`` = k_e / eps_r. Returns the force
    F (ni, 3) (acceleration is F / m) and optionally phi (ni,) with
    U = 1/2 sum phi. With ``linear`` the dielectric grows linearly with
    distance (Table 1 LJC(linear)): Coulomb energy kq q_i q_j / r^2, kq = k_e / D.
    """
    lib = _load()
    x = _f64(x, (-1, 3))
    q, sig, eps = _f64(q), _f64(sig), _f64(eps)
    n = x.shape[0]
    idx, idxp = _idx(idx)
    ni = n if idx is None else idx.shape[0]
    f = np.zeros((ni, 3))
    phi = np.zeros(ni) if potential else None
    lib.oracle_ljc_model(n, _dp(x), _dp(q), _dp(sig), _dp(eps), float(kq), 1 if linear else 0,
                         ni, idxp, _dp(f), _dp(phi))
    return (f, phi) if potential else f


def grav_vjp(x, m, lam, G=1.0, eps=0.0, idx=None):
    """J^T lam for Eq. 1 and the mass derivative: returns (g (n,3), gm (n,)), or
    with ``idx`` only those rows, each gathered on its own (g (len(idx),3), gm)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    m = _f64(m)
    lam = _f64(lam, (-1, 3))
    n = x.shape[0]
    if idx is not None:
        idx, idxp = _idx(idx)
        nk = idx.shape[0]
        g = np.zeros((nk, 3))
        gm = np.zeros(nk)
        lib.oracle_grav_vjp_rows(n, _dp(x), _dp(m), float(G), float(eps) ** 2, _dp(lam), nk,
                                 idxp, _dp(g), _dp(gm))
        return g, gm
    g = np.zeros((n, 3))
    gm = np.zeros(n)
    lib.oracle_grav_vjp(n, _dp(x), _dp(m), float(G), float(eps) ** 2, _dp(lam), _dp(g),
                        _dp(gm))
    return g, gm


def ljc_vjp(x, m, q, types, sig_t, eps_t, lam, kq=COULOMB_K / 80.0, linear=False):
    """J^T lam for a = F/m of the LJC law (constant dielectric, or linear with
    ``linear``: Table 1 LJC(linear), reading C3), with mass and per-type derivatives.

    Returns (g (n,3), gm (n,), gsig (ntypes,), geps (ntypes,)).
    """
    lib = _load()
    x = _f64(x, (-1, 3))
    m, q = _f64(m), _f64(q)
    types = np.ascontiguousarray(np.asarray(types, dtype=np.int32))
    sig_t, eps_t = _f64(sig_t), _f64(eps_t)
    lam = _f64(lam, (-1, 3))
    n = x.shape[0]
    nt = sig_t.shape[0]
    g = np.zeros((n, 3))
    gm = np.zeros(n)
    gs = np.zeros(nt)
    ge = np.zeros(nt)
    lib.oracle_ljc_vjp_model(n, _dp(x), _dp(m), _dp(q),
                             types.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nt,
                             _dp(sig_t), _dp(eps_t), float(kq), 1 if linear else 0, _dp(lam),
                             _dp(g), _dp(gm), _dp(gs), _dp(ge))
    return g, gm, gs, ge


# ---------------------------------------------------------------------------
# Systems: a law plus its parameters, as one object the integrator can call
# ---------------------------------------------------------------------------
class GravSystem:
    """Softened gravity, Eq. 1, with constant G and softening eps."""

    law = "grav"

    def __init__(self, m, G=1.0, eps=0.0):
        self.m = _f64(m)
        self.G = float(G)
        self.eps = float(eps)

    def accel(self, x, potential=False):
        return grav_accel(x, self.m, self.G, self.eps, potential=potential)

    def potential_energy(self, x):
        _, phi = grav_accel(x, self.m, self.G, self.eps, potential=True)
        return 0.5 * float(np.sum(self.m * phi))

    def vjp(self, x, lam):
        """Returns (J^T lam, d/dm (lam . a))."""
        return grav_vjp(x, self.m, lam, self.G, self.eps)


class LJCSystem:
    """LJC(constant) with per-type sigma/epsilon; acceleration a = F / m."""

    law = "ljc"

    def __init__(self, m, q, types, sig_t, eps_t, kq=COULOMB_K / 80.0, linear=False):
        self.linear = bool(linear)
        self.m = _f64(m)
        self.q = _f64(q)
        self.types = np.asarray(types, dtype=np.int32)
        self.sig_t = _f64(sig_t)
        self.eps_t = _f64(eps_t)
        self.kq = float(kq)

    def accel(self, x, potential=False):
        sig = self.sig_t[self.types]
        eps = self.eps_t[self.types]
        out = ljc_force(x, self.q, sig, eps, self.kq, potential=potential, linear=self.linear)
        if potential:
            f, phi = out
            return f / self.m[:, None], phi
        return out / self.m[:, None]

    def potential_energy(self, x):
        sig = self.sig_t[self.types]
        eps = self.eps_t[self.types]
        _, phi = ljc_force(x, self.q, sig, eps, self.kq, potential=True, linear=self.linear)
        return 0.5 * float(np.sum(phi))

    def vjp(self, x, lam):
        """Returns (J^T lam, d/dm, d/dsig_t, d/deps_t) of lam . a."""
        return ljc_vjp(x, self.m, self.q, self.types, self.sig_t, self.eps_t, lam, self.kq,
                       linear=self.linear)


# ---------------------------------------------------------------------------
# Update step of Sec. 1: kick-drift-kick leapfrog (the paper names no integrator)
# ---------------------------------------------------------------------------
def leapfrog(system, x0, v0, dt, nsteps, store=False):
    """Advance (x, v) by ``nsteps`` KDK steps of size ``dt`` in FP64.

    Each step: v += dt/2 a(x); x += dt v; v += dt/2 a(x). Returns (x, v) or,
    with ``store``, lists of all states x_0..x_T and v_0..v_T.
    """
    x = _f64(x0, (-1, 3)).copy()
    v = _f64(v0, (-1, 3)).copy()
    a = system.accel(x)
    xs, vs = [x.copy()], [v.copy()]
    for _ in range(int(nsteps)):
        v = v + 0.5 * dt * a
        x = x + dt * v
        a = system.accel(x)
        v = v + 0.5 * dt * a
        if store:
            xs.append(x.copy())
            vs.append(v.copy())
    if store:
        return xs, vs
    return x, v


def hermite(x0, v0, m, dt, nsteps, G=1.0, eps=0.0, store=False):
    """Fourth-order Hermite predictor-evaluate-correct steps (the integrator
    that consumes Table 1's acceleration and jerk; Makino & Aarseth 1992):
      predict  x_p = x + v dt + a dt^2/2 + j dt^3/6,   v_p = v + a dt + j dt^2/2
      evaluate a_1, j_1 at (x_p, v_p)
      correct  v_1 = v + (a + a_1) dt/2 + (j - j_1) dt^2/12
               x_1 = x + (v + v_1) dt/2 + (a - a_1) dt^2/12
    Returns (x, v) or, with ``store``, lists of all states."""
    x = _f64(x0, (-1, 3)).copy()
    v = _f64(v0, (-1, 3)).copy()
    a, j = grav_jerk(x, v, m, G, eps)
    xs, vs = [x.copy()], [v.copy()]
    for _ in range(int(nsteps)):
        xp = x + v * dt + a * (dt * dt / 2.0) + j * (dt ** 3 / 6.0)
        vp = v + a * dt + j * (dt * dt / 2.0)
        a1, j1 = grav_jerk(xp, vp, m, G, eps)
        v1 = v + (a + a1) * (dt / 2.0) + (j - j1) * (dt * dt / 12.0)
        x1 = x + (v + v1) * (dt / 2.0) + (a - a1) * (dt * dt / 12.0)
        x, v, a, j = x1, v1, a1, j1
        if store:
            xs.append(x.copy())
            vs.append(v.copy())
    if store:
        return xs, vs
    return x, v


def diagnostics(system, x, v):
    """FP64 conserved quantities: dict with K, U, E, P (3,), L (3,)."""
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    m = system.m
    K = 0.5 * float(np.sum(m[:, None] * v * v))
    U = system.potential_energy(x)
    P = np.sum(m[:, None] * v, axis=0)
    L = np.sum(m[:, None] * np.cross(x, v), axis=0)
    return {"K": K, "U": U, "E": K + U, "P": P, "L": L}


# ---------------------------------------------------------------------------
# Reverse-mode KDK (all states stored; no checkpointing needed at oracle sizes)
# ---------------------------------------------------------------------------
def adjoint_leapfrog(system, x0, v0, dt, nsteps, lam_xT, lam_vT=None, xs=None):
    """Gradient of a loss L(x_T, v_T) w.r.t. x_0, v_0 and the law's parameters.

    ``lam_xT`` = dL/dx_T, ``lam_vT`` = dL/dv_T (default 0). The reverse of one
    KDK step (x_n, v_n) -> (x_{n+1}, v_{n+1}), with h = dt/2 and v' the
    half-step velocity, is
        lam_v' = lam_v;     lam_x += h J(x_{n+1})^T lam_v
        lam_v' += dt lam_x
        lam_v  = lam_v';    lam_x += h J(x_n)^T lam_v'
    and every J^T application adds its parameter derivative scaled by h.
    Returns a dict with "x0", "v0", "m" and, for LJC, "sig_t", "eps_t".
    """
    if xs is None:
        xs, _ = leapfrog(system, x0, v0, dt, nsteps, store=True)
    lx = _f64(lam_xT, (-1, 3)).copy()
    lv = np.zeros_like(lx) if lam_vT is None else _f64(lam_vT, (-1, 3)).copy()
    h = 0.5 * dt
    gm = np.zeros(lx.shape[0])
    gs = np.zeros(len(getattr(system, "sig_t", [])))
    ge = np.zeros_like(gs)

    def apply(x, lam, w):
        nonlocal gm, gs, ge
        out = system.vjp(x, lam)
        gm = gm + w * out[1]
        if system.law == "ljc":
            gs = gs + w * out[2]
            ge = ge + w * out[3]
        return w * out[0]

    for n in range(int(nsteps) - 1, -1, -1):
        lx = lx + apply(xs[n + 1], lv, h)
        lv = lv + dt * lx
        lx = lx + apply(xs[n], lv, h)
    res = {"x0": lx, "v0": lv, "m": gm}
    if system.law == "ljc":
        res["sig_t"] = gs
        res["eps_t"] = ge
    return res


def target_loss(x, target):
    """L = (1/N) sum_i |x_i - x*_i|^2 (the adjoint workload's loss)."""
    d = _f64(x, (-1, 3)) - _f64(target, (-1, 3))
    return float(np.sum(d * d)) / d.shape[0]


def target_loss_grad(x, target):
    """dL/dx for :func:`target_loss`."""
    d = _f64(x, (-1, 3)) - _f64(target, (-1, 3))
    return 2.0 * d / d.shape[0]
