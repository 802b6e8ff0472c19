"""The synthetic workloads (seeded, shapes and distributions of the paper's sphere problems).

* sphere_fp64: one sound-hard unit sphere, 128 quadratic elements / 258 nodes, incident
  Gaussian plane-wave pulse along +z (sigma = 0.5), k_m = m/8 (m = 1..64), 1000 observation
  points uniform in volume in the shell 1.05 < r < 3 (seed 1001), 256 time samples.
* spheroid_learned: one sound-hard prolate spheroid, semi-axes (1, 1, 2) with the long axis along
  the propagation direction +z, 1280 elements / 2562 nodes (icosahedral grid, 8 divisions per
  face, mapped onto the exact spheroid), k_m = 20 m / 1024 (m = 1..1024), 256 observation points
  seeded (3001) in the shell between the spheroid scaled by 1.2 and by 2.5, Gaussian sigma = 0.2,
  2048 time samples.
* two_spheres_mixed: two sound-hard unit spheres, 720 elements / 1442 nodes each (N = 2884),
  centres (0, 0, +-1.05) (surface gap 0.1) on the propagation axis, k_m = m/32 (m = 1..512),
  128 x 128 observation grid on the plane z = 0 over [-5, 5]^2, Gaussian sigma = 0.25,
  1024 time samples.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .meshes import Mesh, octa_sphere, ico_sphere, scale_translate, merge_meshes, ellipsoid_from_sphere
from .pulses import gaussian_pulse


@dataclass
class Workload:
    name: str
    mesh: Mesh
    k: np.ndarray            # float64 [Nk], k_m = m * dk, m = 1..Nk
    dk: float
    direction: np.ndarray    # float64 [3], unit propagation direction of the plane wave
    xobs: np.ndarray         # float64 [M, 3]
    pulses: np.ndarray       # float64 [P, Nt] samples of s(t_n)
    Nt: int
    T: float                 # period of the time window = 2*pi / dk


def shell_points(M: int, r0: float, r1: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((M, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    u = rng.random(M)
    r = (r0 ** 3 + u * (r1 ** 3 - r0 ** 3)) ** (1.0 / 3.0)
    return d * r[:, None]


def plane_grid_points(n: int, half: float, z: float = 0.0) -> np.ndarray:
    g = np.linspace(-half, half, n)
    X, Y = np.meshgrid(g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(n * n, z)], axis=1)


def config_sphere_fp64(Nk: int = 64, M: int = 1000, Nt: int = 256, levels: int = 2) -> Workload:
    mesh = octa_sphere(levels, 1.0, bc=0)
    dk = 1.0 / 8.0
    T = 2.0 * np.pi / dk
    k = dk * np.arange(1, Nk + 1, dtype=np.float64)
    xobs = shell_points(M, 1.05, 3.0, seed=1001)
    pulses = gaussian_pulse(Nt, T, sigma=0.5, tc=8.0)[None, :]
    return Workload("sphere_fp64", mesh, k, dk, np.array([0.0, 0.0, 1.0]), xobs, pulses, Nt, T)


def config_two_spheres_mixed(Nk: int = 512, grid: int = 128, Nt: int = 1024, freq: int = 6) -> Workload:
    s = ico_sphere(freq, 1.0, bc=0)
    mesh = merge_meshes([scale_translate(s, 1.0, (0.0, 0.0, -1.05)),
                         scale_translate(s, 1.0, (0.0, 0.0, 1.05))])
    dk = 1.0 / 32.0
    T = 2.0 * np.pi / dk
    k = dk * np.arange(1, Nk + 1, dtype=np.float64)
    xobs = plane_grid_points(grid, 5.0, 0.0)
    pulses = gaussian_pulse(Nt, T, sigma=0.25, tc=8.0)[None, :]
    return Workload("two_spheres_mixed", mesh, k, dk, np.array([0.0, 0.0, 1.0]), xobs, pulses, Nt, T)


def spheroid_shell_points(M: int, axes, s0: float, s1: float, seed: int) -> np.ndarray:
    """Points s * (u * axes) with u uniform on the unit sphere and s uniform in [s0, s1]: outside
    the ellipsoid of those semi-axes when s0 > 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.standard_normal((M, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    s = s0 + (s1 - s0) * rng.random(M)
    return u * np.asarray(axes, dtype=np.float64)[None, :] * s[:, None]


def config_spheroid_learned(Nk: int = 1024, kmax: float = 20.0, freq: int = 8, M: int = 256,
                            Nt: int = 2048) -> Workload:
    axes = (1.0, 1.0, 2.0)
    mesh = ellipsoid_from_sphere(ico_sphere(freq, 1.0, bc=0), axes)
    dk = kmax / Nk
    T = 2.0 * np.pi / dk
    k = dk * np.arange(1, Nk + 1, dtype=np.float64)
    xobs = spheroid_shell_points(M, axes, 1.2, 2.5, seed=3001)
    pulses = gaussian_pulse(Nt, T, sigma=0.2, tc=8.0)[None, :]
    return Workload("spheroid_learned", mesh, k, dk, np.array([0.0, 0.0, 1.0]), xobs, pulses, Nt, T)
