"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself:
library routines (numpy, scipy), closed forms, exact quadrature of monomials, the analytic
sphere series, Green's-identity special solutions and convergence under mesh refinement.
Each test names the passage of the paper whose reading it checks."""
import math
import os

import numpy as np
import pytest

import oracle
import analytic_sphere as an
from workloads import octa_sphere, ico_sphere, shell_points, gaussian_pulse, merge_meshes, scale_translate

D = np.array([0.0, 0.0, 1.0])


# ---------------- quadrature and shape functions (Sec. 3: quadratic elements, Gauss rules) ----
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 16])
def test_gauss_legendre_matches_numpy(n):
    x, w = oracle.gauss_legendre01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, (xr + 1) / 2, atol=2e-15)
    np.testing.assert_allclose(w, wr / 2, atol=2e-15)


def _monomial(a, b):  # exact integral of xi^a eta^b over the reference triangle
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_std_rule_exact_for_polynomials(n):
    xi, eta, w = oracle.rule_std(n)
    assert len(w) == n * n and np.all(w > 0)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            np.testing.assert_allclose(np.sum(w * xi ** a * eta ** b), _monomial(a, b), rtol=1e-13)


@pytest.mark.parametrize("node", range(6))
def test_near_rule_exact_and_collapsed_on_node(node):
    n = 6
    xi, eta, w = oracle.rule_near(n, node)
    assert len(w) == (n * n if node < 3 else 2 * n * n)
    ref = [(0, 0), (1, 0), (0, 1), (0.5, 0), (0.5, 0.5), (0, 0.5)][node]
    # every point strictly inside, none on the collocation node
    assert np.all(np.hypot(xi - ref[0], eta - ref[1]) > 1e-3)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            np.testing.assert_allclose(np.sum(w * xi ** a * eta ** b), _monomial(a, b), rtol=1e-12)


def test_shape_functions_kronecker_and_quadratic_reproduction():
    ref = [(0, 0), (1, 0), (0, 1), (0.5, 0), (0.5, 0.5), (0, 0.5)]
    for b, (x, y) in enumerate(ref):
        N, _, _ = oracle.shape6(x, y)
        np.testing.assert_allclose(N, np.eye(6)[b], atol=1e-15)
    rng = np.random.default_rng(0)
    f = lambda x, y: 1.3 - 0.7 * x + 2.1 * y + 0.4 * x * x - 1.1 * x * y + 0.9 * y * y
    fx = lambda x, y: -0.7 + 0.8 * x - 1.1 * y
    fy = lambda x, y: 2.1 - 1.1 * x + 1.8 * y
    fv = np.array([f(*p) for p in ref])
    for _ in range(20):
        x, y = rng.random(2) * 0.5
        N, dx, dy = oracle.shape6(x, y)
        assert abs(N.sum() - 1) < 1e-15
        assert abs(N @ fv - f(x, y)) < 1e-14
        assert abs(dx @ fv - fx(x, y)) < 1e-13 and abs(dy @ fv - fy(x, y)) < 1e-13


# ---------------- App. B: the surface at infinity (reading: I1 = +4 pi, I2 = 0) ----------------
@pytest.mark.parametrize("k,R", [(1.0, 7.0), (2.5, 31.0)])
def test_appendix_b_surface_at_infinity(k, R):
    """Integrate [dg/dn G - dG/dn g] and the f analogue over a sphere of radius R about x0
    (outward normal) with scipy-free midpoint/Gauss quadrature: the g integral equals +4 pi
    for every R by Green's identity for the regular g, the f integral vanishes."""
    nt = 400
    ct, wt = np.polynomial.legendre.leggauss(nt)  # u = cos(theta) in [-1, 1]
    # g, f depend only on u (k.n0 along the polar axis), so the azimuth integral is 2 pi
    s = k * R * ct
    g, f = np.cos(s), np.sin(s) / k
    dg = -k * np.sin(s) * ct          # grad g . n with n = r/R
    df = np.cos(s) * ct
    G = np.exp(1j * k * R) / R
    dG = np.exp(1j * k * R) * (1j * k * R - 1) / R ** 2
    I1 = 2 * np.pi * R ** 2 * np.sum(wt * (dg * G - dG * g))
    I2 = 2 * np.pi * R ** 2 * np.sum(wt * (df * G - dG * f))
    assert abs(I1 - 4 * np.pi) < 1e-9
    assert abs(I2) < 1e-9


# ---------------- Eq. BRIEF assembly: identities that fix every term -------------------------
def _residuals(mesh, k, u, du, with_4pi):
    H, Gm, al, be = oracle.assemble_raw(mesh, k)
    c = 4 * np.pi if with_4pi else 0.0
    res = H @ u - (c + al) * u - Gm @ du - be * du
    return np.linalg.norm(res) / (4 * np.pi * np.linalg.norm(u))


@pytest.mark.parametrize("k", [1.0, 3.0])
def test_entire_solution_identity_converges(k):
    """u = exp(i k d.x) is regular inside the body, so the row equation without the S_inf term
    must vanish up to discretisation error, at better than second order."""
    errs = []
    for L in (1, 2, 3):
        m = octa_sphere(L)
        u = np.exp(1j * k * m.nodes @ D)
        du = 1j * k * (m.normals @ D) * u
        errs.append(_residuals(m, k, u, du, with_4pi=False))
    assert errs[2] < 2e-4
    assert errs[0] / errs[1] > 7 and errs[1] / errs[2] > 7


@pytest.mark.parametrize("k", [0.0, 1.0, 3.0])
def test_interior_point_source_fixes_infinity_term(k):
    """A point source inside the body is a radiating exterior solution: the full row equation,
    with +4 pi P(x_i) from S_inf, must vanish; with -4 pi it is off by 8 pi P."""
    s = np.array([0.2, -0.1, 0.3])
    errs = []
    for L in (1, 2, 3):
        m = octa_sphere(L)
        r = m.nodes - s
        R = np.linalg.norm(r, axis=1)
        u = np.exp(1j * k * R) / R
        du = np.exp(1j * k * R) * (1j * k * R - 1) * np.einsum("ij,ij->i", r, m.normals) / R ** 3
        errs.append(_residuals(m, k, u, du, with_4pi=True))
        if L == 2:
            H, Gm, al, be = oracle.assemble_raw(m, k)
            wrong = H @ u - (-4 * np.pi + al) * u - Gm @ du - be * du
            assert np.linalg.norm(wrong) / (4 * np.pi * np.linalg.norm(u)) > 1.5
    assert errs[2] < 1e-4
    assert errs[0] / errs[1] > 7 and errs[1] / errs[2] > 7


def test_laplace_limit_linear_solution_identity():
    """k = 0 (the zero-frequency term of Eq. inverseFourier): u = c.x + u0 is harmonic and regular
    inside the body, so the row equation without the S_inf term vanishes up to discretisation
    error.  Its normal derivative c.nu enters through f's limit nu_i.(x - x_i): with f dropped the
    residual stays at 0.27, with f negated at 0.55, at every refinement (measured)."""
    c = np.array([0.3, -0.5, 0.8])
    errs = []
    for L in (1, 2, 3):
        m = octa_sphere(L)
        u = (m.nodes @ c + 0.4).astype(complex)
        du = (m.normals @ c).astype(complex)
        errs.append(_residuals(m, 0.0, u, du, with_4pi=False))
    assert errs[2] < 2e-4
    assert errs[0] / errs[1] > 7 and errs[1] / errs[2] > 7


def test_laplace_limit_is_the_limit_of_the_wavenumber_system():
    """The k = 0 system is the k -> 0 limit of the k > 0 system: every entry of A and b at
    k = 1e-7 agrees with k = 0 to O(k R), for a soft and a hard body."""
    for bc in (0, 1):
        m = octa_sphere(1, bc=bc)
        A0, b0 = oracle.assemble_system(m, 0.0, D)
        A1, b1 = oracle.assemble_system(m, 1e-7, D)
        assert np.abs(A1 - A0).max() <= 1e-6 * np.abs(A0).max()
        if bc == 1:
            assert np.abs(b1 - b0).max() <= 1e-6 * np.abs(b0).max()
        else:
            assert np.abs(b0).max() == 0.0 and np.abs(b1).max() < 1e-5


@pytest.mark.parametrize("a", [1.0, 0.7])
def test_soft_sphere_zero_frequency_closed_form(a):
    """k = 0 exactly, soft sphere of radius a: P_scat = -a/r, so dP/dnu = 1/a on the surface and
    the field is -a/r outside; the discrete solution converges to it under refinement."""
    pts = shell_points(24, 1.3 * a, 3.0 * a, seed=5)
    e_surf, e_field = [], []
    for L in (1, 2, 3):
        m = scale_translate(octa_sphere(L, bc=1), a, (0.0, 0.0, 0.0))
        P, Pn = oracle.solve_frequency(m, 0.0, D)
        np.testing.assert_array_equal(P, -np.ones(m.N))
        e_surf.append(np.abs(Pn - 1.0 / a).max() * a)
        T = oracle.field(m, 0.0, P, Pn, pts)
        ex = -a / np.linalg.norm(pts, axis=1)
        e_field.append(np.abs(T - ex).max() / np.abs(ex).max())
    assert e_surf[1] < 2e-3 and e_field[1] < 1e-3    # measured 9.1e-4, 4.0e-4
    assert e_surf[0] / e_surf[1] > 7 and e_surf[1] / e_surf[2] > 7
    assert e_field[2] < 1e-4                          # measured 3.7e-5


def test_hard_body_zero_frequency_scatters_nothing():
    """k = 0, sound-hard body: the known normal derivative -d.nu ik exp(ik d.x) vanishes, so the
    right-hand side and the scattered field are exactly zero."""
    m = octa_sphere(1, bc=0)
    A, b = oracle.assemble_system(m, 0.0, D)
    assert np.abs(b).max() == 0.0
    P, Pn = oracle.solve_frequency(m, 0.0, D)
    assert np.abs(P).max() == 0.0 and np.abs(Pn).max() == 0.0


def test_two_body_point_sources():
    """Two spheres, one interior source in each: still a radiating exterior solution."""
    from workloads import merge_meshes, scale_translate
    s0 = ico_sphere(2)
    m = merge_meshes([scale_translate(s0, 1.0, (0, 0, -1.05)), scale_translate(s0, 1.0, (0, 0, 1.05))])
    k = 1.5
    src = [np.array([0.1, 0.0, -1.0]), np.array([-0.2, 0.1, 1.2])]
    u = np.zeros(m.N, complex)
    du = np.zeros(m.N, complex)
    for s, amp in zip(src, (1.0, 0.5 - 0.3j)):
        r = m.nodes - s
        R = np.linalg.norm(r, axis=1)
        u += amp * np.exp(1j * k * R) / R
        du += amp * np.exp(1j * k * R) * (1j * k * R - 1) * np.einsum("ij,ij->i", r, m.normals) / R ** 3
    assert _residuals(m, k, u, du, with_4pi=True) < 5e-3


# ---------------- full solve vs the analytic sphere series (Sec. 4, last paragraph) -----------
@pytest.mark.parametrize("k", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("hard", [True, False])
def test_sphere_series_and_refinement(k, hard):
    errs = []
    for L in (1, 2, 3):
        m = octa_sphere(L, bc=0 if hard else 1)
        P, Pn = oracle.solve_frequency(m, k, D)
        if hard:
            ex, got = an.scattered(m.nodes, k, hard=True), P
        else:
            ex, got = an.surface_normal_derivative(m.nodes, k, hard=False), Pn
        errs.append(np.linalg.norm(got - ex) / np.linalg.norm(ex))
    assert errs[1] < 5e-3      # 258 nodes: "better than 2 significant figures"
    assert errs[2] < 4e-4
    assert errs[0] / errs[1] > 7 and errs[1] / errs[2] > 7


def test_soft_sphere_low_frequency_limit():
    """k -> 0 soft sphere: P_scat -> -a/r."""
    m = octa_sphere(2, bc=1)
    k = 1e-3
    P, Pn = oracle.solve_frequency(m, k, D)
    pts = shell_points(20, 1.5, 3.0, seed=3)
    T = oracle.field(m, k, P, Pn, pts)
    np.testing.assert_allclose(T, -1.0 / np.linalg.norm(pts, axis=1), rtol=5e-3, atol=2e-3)


# ---------------- Eq. BRIEFdmn field evaluation ------------------------------------------------
def test_field_reproduces_interior_point_source():
    k = 2.0
    s = np.array([0.2, -0.1, 0.3])
    pts = shell_points(30, 1.05, 3.0, seed=7)
    errs = []
    for L in (1, 2, 3):
        m = octa_sphere(L)
        r = m.nodes - s
        R = np.linalg.norm(r, axis=1)
        G = np.exp(1j * k * R) / R
        dG = np.exp(1j * k * R) * (1j * k * R - 1) * np.einsum("ij,ij->i", r, m.normals) / R ** 3
        T = oracle.field(m, k, G, dG, pts)
        Rp = np.linalg.norm(pts - s, axis=1)
        ex = np.exp(1j * k * Rp) / Rp
        errs.append(np.linalg.norm(T - ex) / np.linalg.norm(ex))
    assert errs[2] < 5e-4 and errs[0] / errs[1] > 5 and errs[1] / errs[2] > 5


def test_field_vs_series_after_solve():
    k = 1.0
    pts = shell_points(30, 1.05, 3.0, seed=8)
    m = octa_sphere(3)
    P, Pn = oracle.solve_frequency(m, k, D)
    T = oracle.field(m, k, P, Pn, pts)
    ex = an.scattered(pts, k, hard=True)
    assert np.linalg.norm(T - ex) / np.linalg.norm(ex) < 1e-3


def test_foot_points_on_sphere():
    m = octa_sphere(2)
    pts = shell_points(50, 1.02, 4.0, seed=5)
    fe, fx, fy = oracle.foot_points(m, pts)
    assert np.all(fe >= 0)
    for p, e, x, y in zip(pts, fe, fx, fy):
        N, dx, dy = oracle.shape6(x, y)
        X = m.nodes[m.elems[e]]
        x0 = N @ X
        t1, t2 = dx @ X, dy @ X
        # the quadratic surface is within O(h^3) of the sphere; the foot point is nearly radial
        assert abs(np.linalg.norm(x0) - 1.0) < 2e-3
        assert abs(np.linalg.norm(p - x0) - (np.linalg.norm(p) - 1.0)) < 3e-3
        if x > 1e-9 and y > 1e-9 and x + y < 1 - 1e-9:  # interior stationary point
            r = p - x0
            assert abs(r @ t1) < 1e-9 * np.linalg.norm(t1) and abs(r @ t2) < 1e-9 * np.linalg.norm(t2)


# ---------------- direct solver ------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 7, 64, 200])
def test_lu_against_numpy(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = oracle.solve(A, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)
    be = np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 1) * np.linalg.norm(x) + np.linalg.norm(b))
    assert be < 10 * n * np.finfo(float).eps


def test_lu_pivot_order_and_singular():
    A = np.array([[1.0, 2.0], [3.0, 4.0]], complex)
    LU, piv = oracle.lu_factor(A)
    assert list(piv) == [1, 1]
    with pytest.raises(RuntimeError):
        oracle.lu_factor(np.zeros((3, 3), complex))


# ---------------- transforms (Eq. inverseFourier convention, Sec. 4 sampling) ------------------
def test_dft_matches_numpy_and_parseval():
    rng = np.random.default_rng(1)
    s = rng.standard_normal(256)
    S = oracle.dft(s)
    np.testing.assert_allclose(S, 256 * np.fft.ifft(s), rtol=1e-12, atol=1e-11)
    assert abs(np.sum(s ** 2) - np.sum(np.abs(S) ** 2) / 256) < 1e-10 * np.sum(s ** 2)


def test_gaussian_spectrum_closed_form():
    Nt, dk, sigma, tc = 256, 1 / 8, 0.5, 8.0
    T = 2 * np.pi / dk
    dt = T / Nt
    S = oracle.dft(gaussian_pulse(Nt, T, sigma, tc))
    w = 2 * np.pi * np.arange(Nt // 2 + 1) / T
    ref = sigma * np.sqrt(2 * np.pi) / dt * np.exp(-(sigma * w) ** 2 / 2) * np.exp(1j * w * tc)
    np.testing.assert_allclose(S[: Nt // 2 + 1], ref, atol=1e-11 * np.abs(ref).max())


def test_synthesis_inverts_and_shifts():
    Nt = 128
    T = 2 * np.pi / 0.25
    s = gaussian_pulse(Nt, T, 1.0, 6.0) - 0.3 * gaussian_pulse(Nt, T, 0.7, 12.0)
    S = oracle.dft(s)
    midx = np.arange(Nt // 2 + 1)
    k = 2 * np.pi * midx / T
    # T_m = 1 at all frequencies reproduces the pulse; T_m = exp(i k_m z) delays it by z (c = 1)
    one = np.ones((len(midx), 1), complex)
    np.testing.assert_allclose(oracle.synthesize(one, midx, S, Nt)[0, 0], s, atol=1e-12)
    j = 5
    z = j * T / Nt
    shift = np.exp(1j * k * z)[:, None]
    np.testing.assert_allclose(oracle.synthesize(shift, midx, S, Nt)[0, 0], np.roll(s, j), atol=1e-12)


def test_causality_of_scattered_pulse():
    """Sec. 4: no scattered field reaches an observation point before the incident pulse has
    touched the body and travelled there.  With the analytic spectra the only leak is the
    spectral truncation at k = 8 (Gaussian spectrum e^-8 there); with the 258-node BIE the
    interior-resonance wavenumbers (j_n zeros near 4.49, 5.76, 6.99) add a ringing tail."""
    Nk, Nt, sigma, tc = 64, 256, 0.5, 8.0
    dk = 1 / 8
    T = 2 * np.pi / dk
    m = octa_sphere(2)
    x = np.array([[0.0, 0.0, -2.5], [1.8, 0.0, 0.5]])
    spectra = np.zeros((Nk, 2), complex)
    for i in range(Nk):
        k = dk * (i + 1)
        P, Pn = oracle.solve_frequency(m, k, D)
        spectra[i] = oracle.field(m, k, P, Pn, x)
    series = np.array([an.scattered(x, dk * (i + 1)) for i in range(Nk)])
    S = oracle.dft(gaussian_pulse(Nt, T, sigma, tc))
    t = np.arange(Nt) * T / Nt
    for spec, bound in ((series, 2e-4), (spectra, 1e-2)):
        p = oracle.synthesize(spec, np.arange(1, Nk + 1), S, Nt)[0]
        for ip, xp in enumerate(x):
            # earliest arrival: the pulse peak reaches z = -1 at t = tc - 1, then travels >= |x| - 1
            t_arr = tc - 1.0 + (np.linalg.norm(xp) - 1.0)
            early = t < t_arr - 6 * sigma
            assert np.abs(p[ip][early]).max() < bound * np.abs(p[ip]).max()
            assert np.abs(p[ip]).max() > 1e-2


def test_assemble_rows_equals_the_system_rows():
    """The row-by-row assembly used for checks at large N is the system's arithmetic, row by row."""
    m = merge_meshes([scale_translate(ico_sphere(2), 0.8, (0, 0, -1.0), bc=1),
                      scale_translate(ico_sphere(2), 1.1, (0.3, 0, 1.3), bc=0)])
    A, b = oracle.assemble_system(m, 2.3, [0.0, 0.0, 1.0])
    rows = np.array([0, 5, 161, m.N - 1])
    Ar, br = oracle.assemble_rows(m, 2.3, [0.0, 0.0, 1.0], rows)
    assert np.array_equal(Ar, A[rows]) and np.array_equal(br, b[rows])


# ---------------- reciprocity of the scattering amplitude (Sec. 2, the scattering problem) ------
def _far_field(mesh, k, P, Pn, xhat):
    """Scattering amplitude in direction xhat from the surface solution: the far-field limit of the
    Green representation of the scattered field, R e^{-ikR} p(R xhat) -> (1/4 pi) sum over elements
    of the surface integral of [P (-ik xhat.nu) - dP/dnu] e^{-ik xhat.y}, evaluated here with its own
    element quadrature (6 x 6 collapsed Gauss-Legendre on each quadratic triangle), independent of
    the oracle's rules."""
    g, gw = np.polynomial.legendre.leggauss(6)
    g, gw = 0.5 * (g + 1.0), 0.5 * gw
    xi = np.repeat(g, 6)
    eta = np.tile(g, 6) * (1.0 - xi)
    w = np.repeat(gw, 6) * np.tile(gw, 6) * (1.0 - xi)
    L = 1.0 - xi - eta
    Nq = np.stack([L * (2 * L - 1), xi * (2 * xi - 1), eta * (2 * eta - 1), 4 * L * xi, 4 * xi * eta, 4 * eta * L], 1)
    dxi = np.stack([1 - 4 * L, 4 * xi - 1, 0 * xi, 4 * (L - xi), 4 * eta, -4 * eta], 1)
    deta = np.stack([1 - 4 * L, 0 * xi, 4 * eta - 1, -4 * xi, 4 * xi, 4 * (L - eta)], 1)
    total = 0.0 + 0.0j
    for el in mesh.elems:
        X = mesh.nodes[el]
        y = Nq @ X
        n = np.cross(dxi @ X, deta @ X)  # |n| = J, oriented into the fluid
        nn = mesh.normals[el]
        n *= np.sign(np.sum(n * (Nq @ nn), axis=1))[:, None]
        ph = np.exp(-1j * k * (y @ xhat))
        total += np.sum(w * (Nq @ P[el] * (-1j * k) * (n @ xhat) - Nq @ Pn[el] * np.linalg.norm(n, axis=1)) * ph)
    return total / (4.0 * np.pi)


def test_scattering_amplitude_reciprocity():
    """Reciprocity f(x, d) = f(-d, -x) of the scattering amplitude (a law of the continuous problem,
    met by the discrete solution to its discretisation error), for a hard and a soft body of
    different sizes, so that no symmetry of the configuration makes it trivial."""
    m = merge_meshes([scale_translate(ico_sphere(3, bc=0), 0.7, (0, 0, -0.9)),
                      scale_translate(ico_sphere(3, bc=1), 0.5, (0.3, 0.2, 0.8))])
    k = 2.0
    d1 = np.array([0.0, 0.0, 1.0])
    d2 = np.array([np.sin(1.1), 0.0, np.cos(1.1)])
    P1, Pn1 = oracle.solve_frequency(m, k, d1)
    P2, Pn2 = oracle.solve_frequency(m, k, d2)
    f12 = _far_field(m, k, P2, Pn2, -d1)  # incidence d2, observed towards -d1
    f21 = _far_field(m, k, P1, Pn1, -d2)  # incidence d1, observed towards -d2
    f11 = _far_field(m, k, P1, Pn1, d2)
    assert abs(f12 - f21) <= 1e-3 * abs(f12), (f12, f21)  # measured 6.5e-5
    assert abs(f11 - f12) > 0.1 * abs(f12)  # a generic pair of amplitudes differs: the pin has teeth


# ---------------- dominant frequencies and Table I (Sec. 4) ------------------------------------
def test_top_frequencies_match_lexsort_with_ties():
    rng = np.random.default_rng(21)
    Nt = 64
    S = rng.standard_normal((3, Nt)) + 1j * rng.standard_normal((3, Nt))
    S[:, 5] = S[:, 9] = 2.5  # a tie: the lower index ranks first
    S[:, 12] = 2.5
    amp = np.abs(S[:, : Nt // 2 + 1]).max(axis=0)
    for K in (0, 1, 2, 3, 7, Nt // 2 + 1):
        order = np.lexsort((np.arange(amp.size), -amp))
        np.testing.assert_array_equal(oracle.top_frequencies(S, K), np.sort(order[:K]))


def _table_one():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_rms.txt")
    rows = [list(map(float, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return np.array(rows)


def rms_percent(pK, pall):
    """Reading of Table I's measure: the RMS over the period's time steps of the difference,
    relative to the largest |p| of the all-frequency signal at that point, in percent."""
    return 100.0 * np.sqrt(((pK - pall) ** 2).mean(axis=-1)) / np.abs(pall).max(axis=-1)


def test_oracle_reproduces_table_one():
    """The paper's own experiment: soft sphere, 1002 nodes, Eq. (pulse) with 2N_c = 4, alpha = 0.1,
    w = 20.1a, 64 frequencies; the field at (0,0,-1.1a) and (0,0,-4a) synthesised from the 5, 10,
    20 dominant frequencies against all 64.  Printed values (tests/golden/table1_rms.txt) within
    30 % (measured 4.35, 4.84 / 1.68, 1.70 / 0.57, 0.55); the kept amplitudes above the printed
    epsilon bounds, which are rounded (the 10th amplitude is 3.497 % of the largest, printed
    "> 3.5 %")."""
    from workloads import config_paper_sphere
    w = config_paper_sphere(bc=1)
    pts = w.xobs[:2]
    S = oracle.dft(w.pulses[0])
    T = np.zeros((len(w.k), 2), complex)
    for i, k in enumerate(w.k):
        P, Pn = oracle.solve_frequency(w.mesh, k, D)
        T[i] = oracle.field(w.mesh, k, P, Pn, pts)
    m_all = np.arange(len(w.k))
    pall = oracle.synthesize(T, m_all, S[None, :], w.Nt)[0]
    amp = np.abs(S[: w.Nt // 2 + 1])
    for K, eps, r11, r40 in _table_one():
        sel = oracle.top_frequencies(S[None, :], int(K))
        assert sel.max() < len(w.k)
        assert amp[sel].min() / amp.max() > 0.98 * eps
        pK = oracle.synthesize(T[sel], sel, S[None, :], w.Nt)[0]
        got = rms_percent(pK, pall)
        np.testing.assert_allclose(got, [r11, r40], rtol=0.3)


# ---------------- input meshes of the paper's other experiments (Sec. 4.1-4.2) -----------------
def test_bowl_mesh_is_a_closed_oriented_surface_of_the_right_volume():
    """The body-of-revolution mesh of Eq. (dish): N = 2E + 2, every directed edge used once and its
    reverse once (a closed, consistently oriented surface), node normals of unit length, and the
    enclosed volume -- by the divergence theorem on the flat sub-triangles -- converging at second
    order to the volume of the solid of revolution, pi int sin^2 t (0.2 sin t + 1.2 sin t cos t) dt
    = 0.8 pi / 3."""
    from collections import Counter
    from workloads import revolution_mesh, bowl_profile
    exact = 0.8 * np.pi / 3.0
    errs = []
    for nt, nph in ((8, 12), (16, 24), (32, 48)):
        m = revolution_mesh(bowl_profile, nt, nph)
        assert m.N == 2 * m.E + 2
        cnt = Counter()
        for e in m.elems:
            for a, b in ((e[0], e[1]), (e[1], e[2]), (e[2], e[0])):
                cnt[(a, b)] += 1
        assert all(c == 1 and cnt[(b, a)] == 1 for (a, b), c in cnt.items())
        np.testing.assert_allclose(np.linalg.norm(m.normals, axis=1), 1.0, rtol=1e-14)
        v = m.nodes[m.elems]
        vol = 0.0
        for t in ((0, 3, 5), (3, 1, 4), (5, 4, 2), (3, 4, 5)):
            a, b, c = v[:, t[0]], v[:, t[1]], v[:, t[2]]
            vol += np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
        errs.append(abs(vol - exact))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5 and errs[2] < 2e-3


def test_bowl_normals_are_perpendicular_to_the_surface():
    """Exact node normals against the tangents of the quadratic elements at their vertices."""
    from workloads import revolution_mesh, bowl_profile
    m = revolution_mesh(bowl_profile, 24, 32)
    worst = 0.0
    for e in m.elems:
        x = m.nodes[e]
        for a, (xi, eta) in enumerate(((0, 0), (1, 0), (0, 1))):
            _, dN1, dN2 = oracle.shape6(xi, eta)
            t1, t2 = dN1 @ x, dN2 @ x
            n = m.normals[e[a]]
            worst = max(worst, abs(n @ t1) / np.linalg.norm(t1), abs(n @ t2) / np.linalg.norm(t2))
    assert worst < 1.2e-2  # measured 8.4e-3 (second order: 3.9e-2 at 12 x 16, 2.2e-3 at 48 x 64)


# ---------------- linear 3-node elements (Sec. 4's cross-check) --------------------------------
def test_shape3_kronecker_and_linear_reproduction():
    ref = [(0, 0), (1, 0), (0, 1)]
    for a, (xi, eta) in enumerate(ref):
        N, _, _ = oracle.shape3(xi, eta)
        np.testing.assert_allclose(N, np.eye(3)[a], atol=0)
    rng = np.random.default_rng(3)
    for _ in range(5):
        xi, eta = rng.random(2) * 0.5
        N, dx, de = oracle.shape3(xi, eta)
        f = np.array([2.0 - 3.0 * x + 0.5 * y for x, y in ref])
        assert abs(N @ f - (2.0 - 3.0 * xi + 0.5 * eta)) < 1e-14
        assert abs(dx @ f + 3.0) < 1e-14 and abs(de @ f - 0.5) < 1e-14


def _linear_residuals(m, k, u, du, with_4pi):
    H, Gm, al, be = oracle.assemble_raw_linear(m, k)
    c = 4 * np.pi if with_4pi else 0.0
    res = H @ u - (c + al) * u - Gm @ du - be * du
    return np.linalg.norm(res) / (4 * np.pi * np.linalg.norm(u))


@pytest.mark.parametrize("k", [0.0, 1.5])
def test_linear_elements_point_source_and_entire_solution(k):
    """Flat elements with linear interpolation: an interior point source satisfies the full row
    equation and exp(i k d.x) (or, at k = 0, a linear function) the one without S_inf, both up to
    a discretisation error that falls at second order; -4 pi instead of +4 pi leaves O(1)."""
    from workloads import uv_sphere_linear
    s = np.array([0.2, -0.1, 0.3])
    e_src, e_ent = [], []
    for nt, nph in ((8, 16), (16, 32), (32, 64)):
        m = uv_sphere_linear(nt, nph)
        r = m.nodes - s
        R = np.linalg.norm(r, axis=1)
        u = np.exp(1j * k * R) / R
        du = np.exp(1j * k * R) * (1j * k * R - 1) * np.einsum("ij,ij->i", r, m.normals) / R ** 3
        e_src.append(_linear_residuals(m, k, u, du, True))
        if nt == 16:
            H, Gm, al, be = oracle.assemble_raw_linear(m, k)
            wrong = H @ u - (-4 * np.pi + al) * u - Gm @ du - be * du
            assert np.linalg.norm(wrong) / (4 * np.pi * np.linalg.norm(u)) > 1.5
        if k > 0:
            v = np.exp(1j * k * m.nodes @ D)
            dv = 1j * k * (m.normals @ D) * v
        else:
            c = np.array([0.3, -0.5, 0.8])
            v = (m.nodes @ c + 0.4).astype(complex)
            dv = (m.normals @ c).astype(complex)
        e_ent.append(_linear_residuals(m, k, v, dv, False))
    for e in (e_src, e_ent):
        assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e
    assert e_src[2] < 5e-3 and e_ent[2] < 5e-3


@pytest.mark.parametrize("hard", [True, False])
def test_linear_elements_sphere_series(hard):
    """Sphere series at k = 1: second-order convergence on latitude-longitude meshes, and the
    paper's 774-element / 389-node mesh within 3 % (measured 2.7 % hard, 2.4 % soft)."""
    from workloads import uv_sphere_linear
    k = 1.0
    errs = []
    for nt, nph in ((8, 16), (16, 32), (32, 64), (10, 43)):
        m = uv_sphere_linear(nt, nph, bc=0 if hard else 1)
        P, Pn = oracle.solve_frequency_linear(m, k, D)
        if hard:
            ex, got = an.scattered(m.nodes, k, hard=True), P
        else:
            ex, got = an.surface_normal_derivative(m.nodes, k, hard=False), Pn
        errs.append(np.linalg.norm(got - ex) / np.linalg.norm(ex))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] < 5e-3 and errs[3] < 3e-2, errs
    assert m.N == 389 and m.E == 774


def test_linear_field_reproduces_interior_point_source():
    from workloads import uv_sphere_linear
    m = uv_sphere_linear(32, 64)
    k = 1.2
    s = np.array([0.1, 0.2, -0.25])
    r = m.nodes - s
    R = np.linalg.norm(r, axis=1)
    P = np.exp(1j * k * R) / R
    Pn = np.exp(1j * k * R) * (1j * k * R - 1) * np.einsum("ij,ij->i", r, m.normals) / R ** 3
    pts = shell_points(10, 1.3, 2.5, seed=7)
    Rp = np.linalg.norm(pts - s, axis=1)
    ex = np.exp(1j * k * Rp) / Rp
    T = oracle.field_linear(m, k, P, Pn, pts)
    assert np.linalg.norm(T - ex) / np.linalg.norm(ex) < 5e-3
