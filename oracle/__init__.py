"""FP64 CPU oracle of semi-Lagrangian Metamorphosis / LDDMM shooting.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline call it; the product path (the CUDA library and its binding) never
does.  It wraps ``meta_oracle.c`` (plain C, FP64) through ctypes.

Functions (arrays are numpy, converted to float64 C-contiguous):

* ``taps(sigma)``                         -- normalised Gaussian taps, r = ceil(3 sigma)
* ``blur(f, sigma)``                      -- K * f, separable, zero padding
* ``diff(f, axis, transpose=False)``      -- central difference D_axis (or its transpose)
* ``interp(F, disp, transpose=False)``    -- S(y) F with y = x + disp (or S(y)^T F)
* ``shoot(I0, p0, T, sigma, mu, rho)``    -- states (I_t, p_t), t=0..T, and u_t
  (``p_update="det"`` on shoot / adjoint / cost_and_grad: p' = p~ det(Id - dt Dv);
  ``scheme="euler"`` / ``"hybrid"`` on shoot / adjoint / cost_and_grad: the other
  integration schemes of Sec. 2.3)
* ``adjoint(I0, p0, gI1, gp1, ...)``      -- gradient of <gI1,I_T>+<gp1,p_T> w.r.t. (I0, p0)
* ``cost_and_grad(I0, J, p0, ...)``       -- Eq. 4 cost (3 terms) and dL/dp0
* ``deformation(I0, p0, T, sigma, mu, rho)`` -- phi_T - Id and det D phi_T (numpy)
* ``jacobian_det(phi)``                   -- det D phi of a map given in coordinates (numpy)
* ``lbfgs_direction(g, S, Y)``              -- the two-loop recursion (numpy)
* ``lbfgs_run(f, x0, ...)``, ``lbfgs_minimize(...)`` -- L-BFGS on any objective, and
  on the Eq. 4 cost (numpy)

Parity pins: see tests/test_oracle_pins.py (closed forms, invariants, dot-product
transpose identities, finite differences, an independent torch re-implementation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "meta_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmeta_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile meta_oracle.c into libmeta_oracle.so (gcc, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_taps.argtypes = [ctypes.c_double, _D, ctypes.c_int]
        lib.oracle_taps.restype = ctypes.c_int
        lib.oracle_blur.argtypes = [ctypes.c_int, _L, ctypes.c_double, _D, _D]
        lib.oracle_diff.argtypes = [ctypes.c_int, _L, ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oracle_interp.argtypes = [ctypes.c_int, _L, _D, ctypes.c_int, _D, _D]
        lib.oracle_shoot.argtypes = [ctypes.c_int, _L, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     _D, _D, _D, _D, _D]
        lib.oracle_shoot_scheme.argtypes = [ctypes.c_int, _L, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, _D, _D, _D, _D, _D]
        lib.oracle_adjoint.argtypes = [ctypes.c_int, _L, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, _D, _D, _D, _D, _D, _D]
        lib.oracle_cost_and_grad.argtypes = [ctypes.c_int, _L, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        for f in ("oracle_blur", "oracle_diff", "oracle_interp", "oracle_shoot",
                  "oracle_shoot_scheme",
                  "oracle_adjoint", "oracle_cost_and_grad"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_D)


def _dims(shape) -> ctypes.Array:
    return (ctypes.c_long * len(shape))(*shape)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def taps(sigma: float) -> np.ndarray:
    """w_k, k = -r..r, r = ceil(3 sigma), sum 1 (the Gaussian RKHS kernel, Sec. 2.1)."""
    buf = np.zeros(4097)
    r = _load().oracle_taps(float(sigma), _ptr(buf), buf.size)
    if r < 0:
        raise ValueError("bad sigma")
    return buf[: 2 * r + 1].copy()


def blur(f, sigma: float) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    _check(_load().oracle_blur(f.ndim, _dims(f.shape), float(sigma), _ptr(f), _ptr(out)), "blur")
    return out


def diff(f, axis: int, transpose: bool = False) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    _check(_load().oracle_diff(f.ndim, _dims(f.shape), int(axis), int(transpose),
                               _ptr(f), _ptr(out)), "diff")
    return out


def interp(F, disp, transpose: bool = False) -> np.ndarray:
    """disp has shape [ndim, *F.shape]: the foot of voxel x is x + disp[:, x]."""
    F = _f64(F)
    disp = _f64(disp)
    assert disp.shape == (F.ndim,) + F.shape
    out = np.empty_like(F)
    _check(_load().oracle_interp(F.ndim, _dims(F.shape), _ptr(disp), int(transpose),
                                 _ptr(F), _ptr(out)), "interp")
    return out


def _pdet(p_update) -> int:
    """Momentum update: 0 / "div" = p~ (1 - dt div v), 1 / "det" = p~ det(Id - dt Dv)."""
    m = {0: 0, 1: 1, "div": 0, "det": 1}
    if p_update not in m:
        raise ValueError("p_update must be 0, 1, 'div' or 'det'")
    return m[p_update]


SCHEMES = {"sl": 0, "euler": 1, "hybrid": 2}


def shoot(I0, p0, T: int, sigma: float, mu: float, rho: float,
          want_u: bool = False, p_update=0,
          scheme: str = "sl") -> Tuple[np.ndarray, np.ndarray, Optional[np.ndarray]]:
    """Returns (I[T+1, ...], p[T+1, ...], u[T, ndim, ...] or None).  scheme: "sl"
    (semi-Lagrangian, the method), "euler" or "hybrid" (the other schemes of Sec. 2.3)."""
    I0, p0 = _f64(I0), _f64(p0)
    shp = I0.shape
    It = np.empty((T + 1,) + shp)
    pt = np.empty((T + 1,) + shp)
    ut = np.empty((T, len(shp)) + shp) if want_u else None
    _check(_load().oracle_shoot_scheme(len(shp), _dims(shp), int(T), float(sigma), float(mu),
                                       float(rho), _pdet(p_update), SCHEMES[scheme], _ptr(I0),
                                       _ptr(p0), _ptr(It), _ptr(pt), _ptr(ut)), "shoot")
    return It, pt, ut


def adjoint(I0, p0, gI1, gp1, T: int, sigma: float, mu: float,
            rho: float, p_update=0, scheme: str = "sl") -> Tuple[np.ndarray, np.ndarray]:
    """Returns (gI0, gp0) for the scalar <gI1, I_T> + <gp1, p_T>."""
    I0, p0, gI1 = _f64(I0), _f64(p0), _f64(gI1)
    gp1 = None if gp1 is None else _f64(gp1)
    shp = I0.shape
    gI0 = np.empty(shp)
    gp0 = np.empty(shp)
    _check(_load().oracle_adjoint(len(shp), _dims(shp), int(T), float(sigma), float(mu),
                                  float(rho), _pdet(p_update), SCHEMES[scheme], _ptr(I0),
                                  _ptr(p0), _ptr(gI1), _ptr(gp1), _ptr(gI0), _ptr(gp0)),
           "adjoint")
    return gI0, gp0


def cost_and_grad(I0, J, p0, T: int, sigma: float, mu: float, rho: float, lam: float,
                  want_grad: bool = True, p_update=0,
                  scheme: str = "sl") -> Tuple[np.ndarray, Optional[np.ndarray]]:
    """Returns (cost3 = [data, lambda*kinetic, lambda*rho*residual], dL/dp0 or None)."""
    I0, J, p0 = _f64(I0), _f64(J), _f64(p0)
    shp = I0.shape
    c3 = np.zeros(3)
    g = np.empty(shp) if want_grad else None
    _check(_load().oracle_cost_and_grad(len(shp), _dims(shp), int(T), float(sigma), float(mu),
                                        float(rho), float(lam), _pdet(p_update), SCHEMES[scheme],
                                        _ptr(I0), _ptr(J), _ptr(p0), _ptr(c3), _ptr(g)),
           "cost_and_grad")
    return c3, g


def jacobian_det(phi) -> np.ndarray:
    """det D phi for a map phi [ndim, *shape] given by its coordinates (axis 0 first).
    D phi_a / D x_e is numpy.gradient along axis e: the central difference inside,
    the one-sided difference on the first and last layer (unit spacing)."""
    phi = _f64(phi)
    nd = phi.shape[0]
    A = np.empty(phi.shape[1:] + (nd, nd))
    for a in range(nd):
        for e in range(nd):
            A[..., a, e] = np.gradient(phi[a], axis=e)
    return np.linalg.det(A)


def deformation(I0, p0, T: int, sigma: float, mu: float, rho: float,
                scheme: str = "sl") -> Tuple[np.ndarray, np.ndarray]:
    """Deformation of the grid along the shot (the deformation grids of Fig. 1-2,
    built from all the v_t of the shot): phi_0 = Id and phi_{t+1} = phi_t o (Id - dt v_t),
    each composition evaluated as S(y) phi_t, the interpolation of phi_t (in
    coordinates) at the clamped foot y of step t, exactly as the image is.
    Returns (phi_T - Id as [ndim, *shape], det D phi_T)."""
    I0 = _f64(I0)
    shp = I0.shape
    nd = len(shp)
    _, _, u = shoot(I0, p0, T, sigma, mu, rho, want_u=True, scheme=scheme)
    ident = np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shp],
                                 indexing="ij"))
    phi = ident.copy()
    dt = 1.0 / T
    for t in range(T):
        disp = -dt * (-rho * u[t])  # y - x = -dt v_t, v_t = -rho u_t
        phi = np.stack([interp(phi[a], disp) for a in range(nd)])
    return phi - ident, jacobian_det(phi)


def lbfgs_direction(g, S, Y, gamma=None) -> np.ndarray:
    """d = -H g by the two-loop recursion (Nocedal & Wright, Numerical Optimization,
    Algorithm 7.4).  S, Y: the stored pairs s_i = x_{i+1} - x_i, y_i = g_{i+1} - g_i,
    oldest first; a pair with s.y <= 1e-12 y.y is skipped.  H_0 = gamma I, gamma by
    default s.y / y.y of the newest usable pair (1 without one)."""
    g = _f64(g)
    use = [(_f64(s), _f64(y)) for s, y in zip(S, Y)
           if (_f64(s) * _f64(y)).sum() > 1e-12 * (_f64(y) ** 2).sum() and (_f64(y) ** 2).sum() > 0]
    q = g.copy()
    alpha = []
    for s, y in reversed(use):
        a = (s * q).sum() / (s * y).sum()
        alpha.append(a)
        q = q - a * y
    if gamma is None:
        gamma = ((use[-1][0] * use[-1][1]).sum() / (use[-1][1] ** 2).sum()) if use else 1.0
    r = gamma * q
    for (s, y), a in zip(use, reversed(alpha)):
        b = (y * r).sum() / (s * y).sum()
        r = r + (a - b) * s
    return -r


def lbfgs_run(f, x0, iters: int, m: int, h0: float):
    """L-BFGS with the rules of the GPU driver, on any objective f(x) -> (L, dL/dx):
    direction -H g over the last m pairs (pairs that fail s.y > 1e-12 y.y stay in the
    window but are skipped); without a usable pair in the window, or when -H g does
    not descend, d = -h0 g / max|g| and the pairs are forgotten (d = 0 at a zero
    gradient, where the run stops); a backtracking line search from step 1, halving
    up to 12 times, takes the first step a with L(x + a d) <= L(x) + 1e-4 a g.d; if
    none passes, the iterate stays and the run stops.  Returns (x, costs [iters + 1],
    margins): margins[k] lists, for every trial of iteration k,
    (L + 1e-4 a g.d - L_trial) / |L| (positive: accepted)."""
    x = _f64(x0).copy()
    L, g = f(x)
    window = []  # (s, y, usable), oldest first, at most m
    hist, margins, stopped = [L], [], False
    for _ in range(iters):
        margins.append([])
        if stopped:
            hist.append(L)
            continue
        usable = [(s, y) for s, y, ok in window if ok]
        d = lbfgs_direction(g, [s for s, _ in usable], [y for _, y in usable]) if usable else None
        if d is None or not ((g * d).sum() < 0):
            gmax = np.abs(g).max()
            d = -(h0 / gmax) * g if gmax > 0 else np.zeros_like(g)
            window = [(s, y, False) for s, y, _ in window]
        gd = (g * d).sum()
        if not gd < 0:  # a stationary point: nothing descends from here
            stopped = True
            hist.append(L)
            continue
        step, acc = 1.0, None
        for _t in range(13):
            xt = x + step * d
            Lt, gt = f(xt)
            margins[-1].append((L + 1e-4 * step * gd - Lt) / max(abs(L), 1e-300))
            if Lt <= L + 1e-4 * step * gd:
                acc = (xt, gt, Lt)
                break
            step *= 0.5
        if acc is None:
            stopped = True
            hist.append(L)
            continue
        xt, gt, Lt = acc
        s, y = xt - x, gt - g
        window.append((s, y, (s * y).sum() > 1e-12 * (y * y).sum() and (y * y).sum() > 0))
        window = window[-m:]
        x, g, L = xt, gt, Lt
        hist.append(L)
    return x, np.array(hist), margins


def lbfgs_minimize(I0, J, p0, T: int, sigma: float, mu: float, rho: float, lam: float,
                   iters: int, m: int, h0: float, p_update=0, scheme: str = "sl"):
    """L-BFGS (`lbfgs_run`'s rules) on the cost of Eq. 4 for one instance, from p0.
    Returns (p, costs [iters + 1], margins) as `lbfgs_run` does."""
    def f(x):
        c, g = cost_and_grad(I0, J, x, T, sigma, mu, rho, lam, p_update=p_update, scheme=scheme)
        return c.sum(), g

    return lbfgs_run(f, p0, iters, m, h0)
