"""Textbook partial-wave series for a plane wave exp(i k z) scattered by a sphere of radius a
centred at the origin (time dependence exp(-i omega t), outgoing h_n = h_n^(1) = j_n + i y_n).

    incident: exp(i k z) = sum_n (2n+1) i^n j_n(kr) P_n(cos t)
    hard:     P_scat = -sum_n (2n+1) i^n [j_n'(ka) / h_n'(ka)] h_n(kr) P_n(cos t)
    soft:     P_scat = -sum_n (2n+1) i^n [j_n(ka)  / h_n(ka) ] h_n(kr) P_n(cos t)

Independent of the oracle: it uses only scipy's spherical Bessel functions and Legendre
polynomials.  Used as a pin of the oracle's full solve and field evaluation.
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def _h(n, x, derivative=False):
    return spherical_jn(n, x, derivative) + 1j * spherical_yn(n, x, derivative)


def scattered(points: np.ndarray, k: float, a: float = 1.0, hard: bool = True, nmax: int | None = None):
    """Scattered pressure at points (|x| >= a) for a unit-amplitude incident exp(i k z)."""
    pts = np.atleast_2d(points)
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 2] / r
    if nmax is None:
        nmax = int(k * a + 20)
    out = np.zeros(pts.shape[0], np.complex128)
    for n in range(nmax + 1):
        if hard:
            c = spherical_jn(n, k * a, True) / _h(n, k * a, True)
        else:
            c = spherical_jn(n, k * a) / _h(n, k * a)
        out += -(2 * n + 1) * (1j ** n) * c * _h(n, k * r) * eval_legendre(n, ct)
    return out


def surface_normal_derivative(points: np.ndarray, k: float, a: float = 1.0, hard: bool = False,
                              nmax: int | None = None):
    """d P_scat / dr on the sphere r = a (the outward normal points into the fluid)."""
    pts = np.atleast_2d(points)
    ct = pts[:, 2] / np.linalg.norm(pts, axis=1)
    if nmax is None:
        nmax = int(k * a + 20)
    out = np.zeros(pts.shape[0], np.complex128)
    for n in range(nmax + 1):
        if hard:
            c = spherical_jn(n, k * a, True) / _h(n, k * a, True)
        else:
            c = spherical_jn(n, k * a) / _h(n, k * a)
        out += -(2 * n + 1) * (1j ** n) * c * k * _h(n, k * a, True) * eval_legendre(n, ct)
    return out


def interior_dirichlet_eigen_ka(kmax: float, nmax: int = 30) -> np.ndarray:
    """Zeros of j_n(ka) in (0, kmax]: wavenumbers at which the exterior BIE has interior
    (fictitious) resonances for a unit sphere."""
    out = []
    xs = np.linspace(1e-3, kmax, 20001)
    for n in range(nmax):
        v = spherical_jn(n, xs)
        idx = np.nonzero(np.sign(v[:-1]) * np.sign(v[1:]) < 0)[0]
        for i in idx:
            lo, hi = xs[i], xs[i + 1]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if np.sign(spherical_jn(n, lo)) * np.sign(spherical_jn(n, mid)) <= 0:
                    hi = mid
                else:
                    lo = mid
            out.append(0.5 * (lo + hi))
    return np.sort(np.array(out))
