"""The synthetic workloads (seeded, shapes and distributions of the paper's sphere problems).

* sphere_fp64: one sound-hard unit sphere, 128 quadratic elements / 258 nodes, incident
  Gaussian plane-wave pulse along +z (sigma = 0.5), k_m = m/8 (m = 1..64), 1000 observation
  points uniform in volume in the shell 1.05 < r < 3 (seed 1001), 256 time samples.
* spheroid_learned: one sound-hard prolate spheroid, semi-axes (1, 1, 2) with the long axis along
  the propagation direction +z, 1280 elements / 2562 nodes (icosahedral grid, 8 divisions per
  face, mapped onto the exact spheroid), k_m = 20 m / 1024 (m = 1..1024), 256 observation points
  seeded (3001) in the shell between the spheroid scaled by 1.2 and by 2.5, Gaussian sigma = 0.2,
  2048 time samples.
* uneven_batch: 64 configurations (seed 4001) of 1-8 sound-hard bodies each -- spheres or
  ellipsoids with semi-axes r (1, U[.5, 1], U[.5, 1]) in a random orientation, r ~ U[0.3, 1.5],
  placed without overlap (gap >= 0.1 between bounding spheres) in the box [0, 10]^3 -- meshed with
  icosahedral grids of about 6 r divisions per face, coarsened so that N stays in [162, 8000];
  256 wavenumbers over (0, 8], 256 seeded points outside the bodies, Gaussian sigma = 0.5,
  512 time samples.
* lattice_large: a 4 x 4 x 2 lattice of sound-soft spheres of radius 0.5 (320 elements / 642 nodes
  each, N = 20544), centres 1.2 (i - 1.5, j - 1.5, l - 0.5), k_m = 24 m / 2048 (ka <= 12), 256 x 256
  observation grid on z = 0 over [-4, 4]^2, eight pulses (Gaussian, Ricker, three Gaussian-modulated
  sinusoids, three seeded random band-limited), 4096 time samples.
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


def _random_rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def uneven_configuration(index: int, seed: int = 4001, n_max: int = 8000):
    """Configuration `index` of the uneven batch: (mesh, body list) -- see the module docstring."""
    rng = np.random.Generator(np.random.PCG64([seed, index]))
    nb = int(rng.integers(1, 9))
    bodies = []
    for _ in range(nb):
        r = float(rng.uniform(0.3, 1.5))
        ell = bool(rng.random() < 0.5)
        axes = (r, r * float(rng.uniform(0.5, 1.0)), r * float(rng.uniform(0.5, 1.0))) if ell else (r, r, r)
        rot = _random_rotation(rng) if ell else np.eye(3)
        for _attempt in range(1000):
            c = rng.uniform(r, 10.0 - r, 3)
            if all(np.linalg.norm(c - b["c"]) >= r + b["r"] + 0.1 for b in bodies):
                bodies.append({"r": r, "axes": axes, "rot": rot, "c": c})
                break
    divs = [max(2, int(round(6.0 * b["r"]))) for b in bodies]
    while sum(40 * n * n + 2 for n in divs) > n_max:
        i = int(np.argmax(divs))
        divs[i] -= 1
    meshes = []
    for b, n in zip(bodies, divs):
        m = ellipsoid_from_sphere(ico_sphere(n, 1.0, bc=0), b["axes"])
        meshes.append(scale_translate(m, 1.0, b["c"], rot=b["rot"]))
    return merge_meshes(meshes), bodies


def outside_points(M: int, bodies, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    while len(pts) < M:
        p = rng.uniform(0.0, 10.0, 3)
        if all(np.linalg.norm(p - b["c"]) > 1.1 * b["r"] + 0.05 for b in bodies):
            pts.append(p)
    return np.array(pts)


def config_uneven_batch(n_configs: int = 64, Nk: int = 256, M: int = 256, Nt: int = 512):
    """List of Workloads, one per configuration, sharing the wavenumber grid and the pulse."""
    dk = 8.0 / Nk
    T = 2.0 * np.pi / dk
    k = dk * np.arange(1, Nk + 1, dtype=np.float64)
    pulse = gaussian_pulse(Nt, T, sigma=0.5, tc=8.0)[None, :]
    out = []
    for i in range(n_configs):
        mesh, bodies = uneven_configuration(i)
        xobs = outside_points(M, bodies, seed=4001 * 1000 + i)
        out.append(Workload(f"uneven_{i}", mesh, k, dk, np.array([0.0, 0.0, 1.0]), xobs, pulse, Nt, T))
    return out


def config_lattice_large(Nk: int = 2048, grid: int = 256, Nt: int = 4096, freq: int = 4) -> Workload:
    s = ico_sphere(freq, 1.0, bc=1)
    bodies = []
    for i in range(4):
        for j in range(4):
            for l in range(2):
                c = (1.2 * (i - 1.5), 1.2 * (j - 1.5), 1.2 * (l - 0.5))
                bodies.append(scale_translate(s, 0.5, c, bc=1))
    mesh = merge_meshes(bodies)
    kmax = 24.0
    dk = kmax / Nk
    T = 2.0 * np.pi / dk
    k = dk * np.arange(1, Nk + 1, dtype=np.float64)
    xobs = plane_grid_points(grid, 4.0, 0.0)
    from .pulses import gaussian_pulse as gp, ricker_pulse, modulated_gaussian
    sig = 1.0 / 12.0
    rows = [gp(Nt, T, sigma=2.0 * sig, tc=4.0), ricker_pulse(Nt, T, kp=8.0, tc=4.0)]
    for kc in (6.0, 12.0, 18.0):
        rows.append(modulated_gaussian(Nt, T, kc=kc, sigma=0.5, tc=4.0))
    # seeded random band-limited signals: sums of the window's harmonics up to angular frequency
    # 20 with normal amplitudes and phases under a cos^2 taper
    rng = np.random.Generator(np.random.PCG64(5001))
    t = np.arange(Nt, dtype=np.float64) * (T / Nt)
    m = np.arange(1, int(20.0 * T / (2.0 * np.pi)) + 1)
    w = 2.0 * np.pi * m / T
    taper = np.cos(0.5 * np.pi * w / 20.0) ** 2
    for _ in range(3):
        amp = rng.standard_normal(m.size) * taper
        ph = rng.uniform(0.0, 2.0 * np.pi, m.size)
        rows.append(np.cos(np.outer(t, w) + ph) @ amp / np.sqrt(m.size))
    pulses = np.stack(rows)
    return Workload("lattice_large", mesh, k, dk, np.array([0.0, 0.0, 1.0]), xobs, pulses, Nt, T)


def config_paper_sphere(bc: int = 1, Nc2: int = 4, alpha: float = 0.1, width: float = 20.1, Nf: int = 128,
                        freq: int = 5, grid: int = 80, half: float = 10.0) -> Workload:
    """The paper's own sphere experiment (Sec. 4): a unit sphere (soft, bc = 1, or hard, bc = 0)
    meshed with 500 quadratic elements / 1002 nodes (icosahedral grid, 5 divisions per face); the
    incident pulse of Eq. (pulse) with 2 N_c = Nc2 cycles modulated by exp(-alpha |tau|) in a window
    of width w = 20.1 a, so k_0 a = 8 pi N_c a / w, sampled at N_f = 128 points of the period
    T = w / c; the 64 frequencies k_m = 2 pi m / w, m = 0 .. 63 (m = 0 included: S_0 vanishes for
    this odd pulse, the zero-frequency solve costs one wavenumber).  Observation points: the two
    points of Table I, (0, 0, -1.1 a) and (0, 0, -4 a), then the 80 x 80 grid of the snapshots in the
    y-z plane over [-10 a, 10 a]^2 without the points inside the sphere (r < 1.02 a)."""
    mesh = ico_sphere(freq, 1.0, bc=bc)
    from .pulses import paper_sine_pulse
    T = width
    k0 = 8.0 * np.pi * (Nc2 / 2.0) / width
    pulses = paper_sine_pulse(Nf, T, k0, Nc2, alpha, 0.0)[None, :]
    dk = 2.0 * np.pi / width
    k = dk * np.arange(0, Nf // 2, dtype=np.float64)
    g = np.linspace(-half, half, grid)
    Y, Z = np.meshgrid(g, g, indexing="ij")
    yz = np.stack([np.zeros(grid * grid), Y.ravel(), Z.ravel()], axis=1)
    yz = yz[np.linalg.norm(yz, axis=1) >= 1.02]
    xobs = np.concatenate([np.array([[0.0, 0.0, -1.1], [0.0, 0.0, -4.0]]), yz])
    return Workload(f"paper_sphere_{'soft' if bc else 'hard'}", mesh, k, dk, np.array([0.0, 0.0, 1.0]), xobs,
                    pulses, Nf, T)



def _yz_grid(n: int, half: float, centre=(0.0, 0.0)) -> np.ndarray:
    g = np.linspace(-half, half, n)
    Y, Z = np.meshgrid(g + centre[0], g + centre[1], indexing="ij")
    return np.stack([np.zeros(n * n), Y.ravel(), Z.ravel()], axis=1)


def config_paper_two_spheres(Nc2: int = 10, alpha: float = 0.1, width: float = 20.1, Nf: int = 128,
                             freq: int = 5, grid: int = 80, half: float = 10.0) -> Workload:
    """Sec. 4.1, Fig. 6: two sound-hard unit spheres 3a apart between centres along the propagation
    direction (centres (0, 0, -1.5) and (0, 0, 1.5)), 1002 nodes each (N = 2004); the pulse of
    Eq. (pulse) with 2N_c = 10 cycles, alpha = 0.1, w = 20.1a (k_0 a = 40 pi / 20.1), N_f = 128, the
    64 frequencies k_m = 2 pi m / w; observation points on the 80 x 80 y-z grid over [-10a, 10a]^2
    and on a finer 61 x 61 grid over [-1.5a, 1.5a] x [-3a, 3a] around the pair, outside both spheres
    by at least 0.02a."""
    s = ico_sphere(freq, 1.0, bc=0)
    mesh = merge_meshes([scale_translate(s, 1.0, (0.0, 0.0, -1.5)), scale_translate(s, 1.0, (0.0, 0.0, 1.5))])
    from .pulses import paper_sine_pulse
    T = width
    k0 = 8.0 * np.pi * (Nc2 / 2.0) / width
    pulses = paper_sine_pulse(Nf, T, k0, Nc2, alpha, 0.0)[None, :]
    dk = 2.0 * np.pi / width
    k = dk * np.arange(0, Nf // 2, dtype=np.float64)
    g = np.linspace(-1.5, 1.5, 61)
    Y, Z = np.meshgrid(g, 2.0 * g, indexing="ij")
    fine = np.stack([np.zeros(Y.size), Y.ravel(), Z.ravel()], axis=1)
    pts = np.concatenate([_yz_grid(grid, half), fine])
    keep = np.ones(len(pts), bool)
    for cz in (-1.5, 1.5):
        keep &= np.linalg.norm(pts - np.array([0.0, 0.0, cz]), axis=1) >= 1.02
    return Workload("paper_two_spheres", mesh, k, dk, np.array([0.0, 0.0, 1.0]), pts[keep], pulses, Nf, T)


def bowl_inside(points: np.ndarray, tilt: float = 0.15 * np.pi, margin: float = 0.0) -> np.ndarray:
    """True where a point lies inside the bowl body of Eq. (dish) (axis tilted by `tilt` about x),
    or within `margin` of it along the axis direction."""
    c, s = np.cos(tilt), np.sin(tilt)
    axis = np.array([0.0, s, c])
    eta = points @ axis
    rho = np.linalg.norm(points - eta[:, None] * axis[None, :], axis=1)
    r = np.clip(rho, 0.0, 1.0)
    half = 0.2 * np.sqrt(1.0 - r * r)
    mid = -0.6 * r * r
    return (rho < 1.0 + margin) & (eta > mid - half - margin) & (eta < mid + half + margin)


def config_paper_bowl(Nc2: int = 6, alpha: float = 0.001, width: float = 20.1, Nf: int = 128,
                      n_theta: int = 48, n_phi: int = 48, grid: int = 81, half: float = 2.0) -> Workload:
    """Sec. 4.2, Figs. 7-8: the sound-hard bowl of Eq. (dish) (the closed curve xi = sin t,
    eta = 0.2 cos t - 0.6 sin^2 t rotated about the eta axis), its axis turned 0.15 pi away from the
    propagation direction +z, meshed by revolution (48 rings x 48 azimuths: E = 4512, N = 9026); the
    pulse of Eq. (pulse) with 2N_c = 6, alpha = 0.001, w = 20.1a (k_0 a = 24 pi / 20.1), N_f = 128,
    64 frequencies; observation points on an 81 x 81 y-z grid over [-2a, 2a]^2 (the plane that
    holds the tilted axis) outside the body by at least 0.02a, and on the 80 x 80 grid of the
    snapshots over [-10a, 10a]^2."""
    from .meshes import bowl_mesh
    from .pulses import paper_sine_pulse
    mesh = bowl_mesh(n_theta, n_phi)
    T = width
    k0 = 8.0 * np.pi * (Nc2 / 2.0) / width
    pulses = paper_sine_pulse(Nf, T, k0, Nc2, alpha, 0.0)[None, :]
    dk = 2.0 * np.pi / width
    k = dk * np.arange(0, Nf // 2, dtype=np.float64)
    pts = np.concatenate([_yz_grid(grid, half), _yz_grid(80, 10.0)])
    pts = pts[~bowl_inside(pts, margin=0.02)]
    return Workload("paper_bowl", mesh, k, dk, np.array([0.0, 0.0, 1.0]), pts, pulses, Nf, T)
