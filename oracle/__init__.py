"""Python view of the CPU FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg are the only callers.  The product library never imports this package, and this package
imports nothing from the product.  Each wrapper documents the passage of the paper it restates
(see oracle.h for the equations).

Parity status of each function (what pins it, in tests/test_oracle_pins.py):
  gauss_legendre01, rule_std, rule_near   pinned: numpy leggauss, exact monomial integrals
  shape6                                  pinned: Kronecker property, quadratic reproduction
  assemble_raw / assemble_system          pinned: entire-solution identity, interior point source,
                                          Appendix-B I1 = +4 pi, convergence order
  lu_factor / lu_solve                    pinned: numpy.linalg.solve, backward error
  foot_points                             pinned: sphere closest point is radial projection
  field                                   pinned: interior point source reproduced, sphere series after a solve
  dft / synthesize                        pinned: numpy FFT, Gaussian closed form, Parseval
  top_frequencies                         pinned: numpy lexsort with ties; Table I of the paper
  *_linear (3-node elements)              pinned: linear reproduction, entire-solution identity and
                                          point source at second order, sphere series at 389 nodes
  full solve                              pinned: analytic rigid/soft sphere partial-wave series;
                                          k = 0: soft sphere -a/r, harmonic linear identity, limit k -> 0
  mlp_features                            pinned: closed-form values at chosen nodes
  mlp_forward / mlp_loss                  pinned: zero-weight and single-path closed forms
  mlp_loss_grad                           pinned: central finite differences of mlp_loss
  adam_step                               pinned: first step moves every parameter by lr*sign(g)
(the mlp_* functions restate the learned warm start of the frequency sweep, which is not part of
the paper's method; its definition is written out at the top of mlp.c)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C11, OpenMP) into oracle/liboracle.so."""
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "mlp.c")]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(f) for f in deps):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        c_dp, c_ip = ctypes.c_void_p, ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "or_gauss_legendre01": [i32, c_dp, c_dp],
            "or_rule_std": [i32, c_dp, c_dp, c_dp],
            "or_rule_near": [i32, i32, c_dp, c_dp, c_dp],
            "or_assemble_raw": [c_dp, i64, c_ip, i64, c_dp, dbl, i32, i32, c_dp, c_dp, c_dp, c_dp],
            "or_assemble_system": [c_dp, i64, c_ip, i64, c_dp, c_ip, dbl, c_dp, i32, i32, c_dp, c_dp],
            "or_lu_factor": [i64, c_dp, c_ip],
            "or_lu_solve": [i64, c_dp, c_ip, c_dp],
            "or_surface_fields": [c_dp, i64, c_dp, c_ip, dbl, c_dp, c_dp, c_dp, c_dp],
            "or_foot_points": [c_dp, i64, c_ip, i64, c_dp, i64, c_ip, c_dp, c_dp],
            "or_field": [c_dp, i64, c_ip, i64, dbl, i32, c_dp, c_dp, c_dp, i64, c_ip, c_dp, c_dp, c_dp],
            "or_dft": [i64, c_dp, c_dp],
            "or_synthesize": [i64, i64, c_dp, c_ip, i64, i64, c_dp, c_dp],
            "or_top_frequencies": [i64, i64, c_dp, i64, c_ip],
            "or_assemble_raw_linear": [c_dp, i64, c_ip, i64, c_dp, dbl, i32, i32, c_dp, c_dp, c_dp, c_dp],
            "or_assemble_system_linear": [c_dp, i64, c_ip, i64, c_dp, c_ip, dbl, c_dp, i32, i32, c_dp, c_dp],
            "or_foot_points_linear": [c_dp, i64, c_ip, i64, c_dp, i64, c_ip, c_dp, c_dp],
            "or_field_linear": [c_dp, i64, c_ip, i64, dbl, i32, c_dp, c_dp, c_dp, i64, c_ip, c_dp, c_dp, c_dp],
            "or_assemble_rows": [c_dp, i64, c_ip, i64, c_dp, c_ip, dbl, c_dp, i32, i32, c_dp, i64, c_dp, c_dp],
            "or_mlp_features": [c_dp, c_dp, i64, c_dp, i64, c_dp, c_dp, dbl, dbl, c_dp],
            "or_mlp_forward": [c_dp, c_dp, i64, c_dp],
            "or_mlp_loss_grad": [c_dp, c_dp, c_dp, i64, c_dp, c_dp],
            "or_mlp_loss": [c_dp, c_dp, c_dp, i64, c_dp],
            "or_adam_step": [i64, c_dp, c_dp, c_dp, c_dp, i64, dbl, dbl, dbl, dbl],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.or_shape6.argtypes = [dbl, dbl, c_dp, c_dp, c_dp]
        lib.or_shape6.restype = None
        lib.or_shape3.argtypes = [dbl, dbl, c_dp, c_dp, c_dp]
        lib.or_shape3.restype = None
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_mlp_param_count.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return int(_load().or_num_threads())


def gauss_legendre01(n: int):
    x, w = np.zeros(n), np.zeros(n)
    _check(_load().or_gauss_legendre01(n, _p(x), _p(w)), "gauss_legendre01")
    return x, w


def shape6(xi: float, eta: float):
    N, dx, de = np.zeros(6), np.zeros(6), np.zeros(6)
    _load().or_shape6(xi, eta, _p(N), _p(dx), _p(de))
    return N, dx, de


def shape3(xi: float, eta: float):
    N, dx, de = np.zeros(3), np.zeros(3), np.zeros(3)
    _load().or_shape3(xi, eta, _p(N), _p(dx), _p(de))
    return N, dx, de


def rule_std(n: int):
    xi, eta, w = np.zeros(n * n), np.zeros(n * n), np.zeros(n * n)
    c = _load().or_rule_std(n, _p(xi), _p(eta), _p(w))
    return xi[:c], eta[:c], w[:c]


def rule_near(n: int, a: int):
    xi, eta, w = np.zeros(2 * n * n), np.zeros(2 * n * n), np.zeros(2 * n * n)
    c = _load().or_rule_near(n, a, _p(xi), _p(eta), _p(w))
    if c < 0:
        raise ValueError("bad near rule")
    return xi[:c], eta[:c], w[:c]


def _mesh_arrays(mesh):
    return (np.ascontiguousarray(mesh.nodes, np.float64), np.ascontiguousarray(mesh.elems, np.int32),
            np.ascontiguousarray(mesh.normals, np.float64), np.ascontiguousarray(mesh.bc, np.uint8))


def assemble_raw(mesh, k: float, ng: int = 4, ng_near: int = 6):
    """H, Gm (N x N), alpha, beta (N) of Eq. BRIEF (Sec. 3, App. A)."""
    nodes, elems, normals, _ = _mesh_arrays(mesh)
    N, E = nodes.shape[0], elems.shape[0]
    H = np.zeros((N, N), np.complex128)
    Gm = np.zeros((N, N), np.complex128)
    al = np.zeros(N, np.complex128)
    be = np.zeros(N, np.complex128)
    _check(_load().or_assemble_raw(_p(nodes), N, _p(elems), E, _p(normals), float(k), ng, ng_near,
                                   _p(H), _p(Gm), _p(al), _p(be)), "assemble_raw")
    return H, Gm, al, be


def assemble_system(mesh, k: float, direction, ng: int = 4, ng_near: int = 6):
    """A, b of the scattered-field system (Eq. BRIEF + App. B + the Sec. 4 BCs)."""
    nodes, elems, normals, bc = _mesh_arrays(mesh)
    d = np.ascontiguousarray(direction, np.float64)
    N, E = nodes.shape[0], elems.shape[0]
    A = np.zeros((N, N), np.complex128)
    b = np.zeros(N, np.complex128)
    _check(_load().or_assemble_system(_p(nodes), N, _p(elems), E, _p(normals), _p(bc), float(k), _p(d),
                                      ng, ng_near, _p(A), _p(b)), "assemble_system")
    return A, b


def assemble_rows(mesh, k: float, direction, rows, ng: int = 4, ng_near: int = 6):
    """Selected rows of the system of assemble_system (same arithmetic, row by row)."""
    nodes, elems, normals, bc = _mesh_arrays(mesh)
    d = np.ascontiguousarray(direction, np.float64)
    rows = np.ascontiguousarray(rows, np.int64)
    N, E = nodes.shape[0], elems.shape[0]
    A = np.zeros((rows.shape[0], N), np.complex128)
    b = np.zeros(rows.shape[0], np.complex128)
    _check(_load().or_assemble_rows(_p(nodes), N, _p(elems), E, _p(normals), _p(bc), float(k), _p(d), ng, ng_near,
                                    _p(rows), rows.shape[0], _p(A), _p(b)), "assemble_rows")
    return A, b


def lu_factor(A: np.ndarray):
    LU = np.ascontiguousarray(A, np.complex128).copy()
    n = LU.shape[0]
    piv = np.zeros(n, np.int64)
    _check(_load().or_lu_factor(n, _p(LU), _p(piv)), "lu_factor")
    return LU, piv


def lu_solve(LU: np.ndarray, piv: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(b, np.complex128).copy()
    _check(_load().or_lu_solve(LU.shape[0], _p(LU), _p(piv), _p(x)), "lu_solve")
    return x


def solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    LU, piv = lu_factor(A)
    return lu_solve(LU, piv, b)


def surface_fields(mesh, k: float, direction, x: np.ndarray):
    nodes, _, normals, bc = _mesh_arrays(mesh)
    d = np.ascontiguousarray(direction, np.float64)
    N = nodes.shape[0]
    P = np.zeros(N, np.complex128)
    Pn = np.zeros(N, np.complex128)
    xx = np.ascontiguousarray(x, np.complex128)
    _check(_load().or_surface_fields(_p(nodes), N, _p(normals), _p(bc), float(k), _p(d), _p(xx),
                                     _p(P), _p(Pn)), "surface_fields")
    return P, Pn


def solve_frequency(mesh, k: float, direction, ng: int = 4, ng_near: int = 6):
    """One frequency solve: assemble, factor, solve; returns (P, dP/dnu) on the surface."""
    A, b = assemble_system(mesh, k, direction, ng, ng_near)
    x = solve(A, b)
    return surface_fields(mesh, k, direction, x)


def foot_points(mesh, xp: np.ndarray):
    nodes, elems, _, _ = _mesh_arrays(mesh)
    xp = np.ascontiguousarray(xp, np.float64)
    M = xp.shape[0]
    fe = np.zeros(M, np.int32)
    fx = np.zeros(M)
    fy = np.zeros(M)
    _check(_load().or_foot_points(_p(nodes), nodes.shape[0], _p(elems), elems.shape[0], _p(xp), M,
                                  _p(fe), _p(fx), _p(fy)), "foot_points")
    return fe, fx, fy


def field(mesh, k: float, P: np.ndarray, Pn: np.ndarray, xp: np.ndarray, foot=None, ng: int = 4):
    """Scattered field at observation points, Eq. BRIEFdmn (S-only form)."""
    nodes, elems, _, _ = _mesh_arrays(mesh)
    xp = np.ascontiguousarray(xp, np.float64)
    if foot is None:
        foot = foot_points(mesh, xp)
    fe, fx, fy = (np.ascontiguousarray(a) for a in foot)
    M = xp.shape[0]
    T = np.zeros(M, np.complex128)
    P = np.ascontiguousarray(P, np.complex128)
    Pn = np.ascontiguousarray(Pn, np.complex128)
    _check(_load().or_field(_p(nodes), nodes.shape[0], _p(elems), elems.shape[0], float(k), ng, _p(P),
                            _p(Pn), _p(xp), M, _p(fe), _p(fx), _p(fy), _p(T)), "field")
    return T


# ---- linear 3-node elements (Sec. 4's cross-check): mesh.elems is [E][3] ---------------------
def assemble_raw_linear(mesh, k: float, ng: int = 4, ng_near: int = 6):
    nodes, elems, normals, _ = _mesh_arrays(mesh)
    N, E = nodes.shape[0], elems.shape[0]
    H = np.zeros((N, N), np.complex128)
    Gm = np.zeros((N, N), np.complex128)
    al = np.zeros(N, np.complex128)
    be = np.zeros(N, np.complex128)
    _check(_load().or_assemble_raw_linear(_p(nodes), N, _p(elems), E, _p(normals), float(k), ng, ng_near,
                                          _p(H), _p(Gm), _p(al), _p(be)), "assemble_raw_linear")
    return H, Gm, al, be


def assemble_system_linear(mesh, k: float, direction, ng: int = 4, ng_near: int = 6):
    nodes, elems, normals, bc = _mesh_arrays(mesh)
    d = np.ascontiguousarray(direction, np.float64)
    N, E = nodes.shape[0], elems.shape[0]
    A = np.zeros((N, N), np.complex128)
    b = np.zeros(N, np.complex128)
    _check(_load().or_assemble_system_linear(_p(nodes), N, _p(elems), E, _p(normals), _p(bc), float(k), _p(d),
                                             ng, ng_near, _p(A), _p(b)), "assemble_system_linear")
    return A, b


def solve_frequency_linear(mesh, k: float, direction, ng: int = 4, ng_near: int = 6):
    A, b = assemble_system_linear(mesh, k, direction, ng, ng_near)
    return surface_fields(mesh, k, direction, solve(A, b))


def foot_points_linear(mesh, xp: np.ndarray):
    nodes, elems, _, _ = _mesh_arrays(mesh)
    xp = np.ascontiguousarray(xp, np.float64)
    M = xp.shape[0]
    fe, fx, fy = np.zeros(M, np.int32), np.zeros(M), np.zeros(M)
    _check(_load().or_foot_points_linear(_p(nodes), nodes.shape[0], _p(elems), elems.shape[0], _p(xp), M,
                                         _p(fe), _p(fx), _p(fy)), "foot_points_linear")
    return fe, fx, fy


def field_linear(mesh, k: float, P: np.ndarray, Pn: np.ndarray, xp: np.ndarray, ng: int = 4):
    nodes, elems, _, _ = _mesh_arrays(mesh)
    xp = np.ascontiguousarray(xp, np.float64)
    fe, fx, fy = foot_points_linear(mesh, xp)
    M = xp.shape[0]
    T = np.zeros(M, np.complex128)
    P = np.ascontiguousarray(P, np.complex128)
    Pn = np.ascontiguousarray(Pn, np.complex128)
    _check(_load().or_field_linear(_p(nodes), nodes.shape[0], _p(elems), elems.shape[0], float(k), ng, _p(P),
                                   _p(Pn), _p(xp), M, _p(fe), _p(fx), _p(fy), _p(T)), "field_linear")
    return T


def dft(s: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(s, np.float64)
    S = np.zeros(s.shape[0], np.complex128)
    _check(_load().or_dft(s.shape[0], _p(s), _p(S)), "dft")
    return S


def synthesize(T: np.ndarray, midx: np.ndarray, S: np.ndarray, Nt: int) -> np.ndarray:
    """p[P][M][Nt] from T[Nk][M] (frequency index midx[r] per row) and pulse spectra S[P][Nt]."""
    T = np.ascontiguousarray(T, np.complex128)
    midx = np.ascontiguousarray(midx, np.int64)
    S = np.ascontiguousarray(np.atleast_2d(S), np.complex128)
    Nk, M = T.shape
    P = S.shape[0]
    out = np.zeros((P, M, Nt))
    _check(_load().or_synthesize(Nk, M, _p(T), _p(midx), P, Nt, _p(S), _p(out)), "synthesize")
    return out


def top_frequencies(S: np.ndarray, K: int) -> np.ndarray:
    """The K frequency indices m (0 <= m <= Nt/2) of largest max over pulses |S[p][m]| (Sec. 4,
    Table I), ties to the lower m, ascending.  S [P][Nt] full spectra (as dft returns them)."""
    S = np.ascontiguousarray(np.atleast_2d(S), np.complex128)
    out = np.zeros(int(K), np.int64)
    _check(_load().or_top_frequencies(S.shape[0], S.shape[1], _p(S), int(K), _p(out)), "top_frequencies")
    return out


# ---- learned warm start (not part of the paper's method; defined at the top of mlp.c) --------
MLP_IN, MLP_WIDTH, MLP_OUT = 64, 256, 2


def mlp_param_count() -> int:
    return int(_load().or_mlp_param_count())


def mlp_param_slices() -> dict:
    """Named views into the flat parameter vector: W1 b1 W2 b2 W3 b3 W4 b4."""
    shapes = [("W1", (MLP_WIDTH, MLP_IN)), ("b1", (MLP_WIDTH,)), ("W2", (MLP_WIDTH, MLP_WIDTH)),
              ("b2", (MLP_WIDTH,)), ("W3", (MLP_WIDTH, MLP_WIDTH)), ("b3", (MLP_WIDTH,)),
              ("W4", (MLP_OUT, MLP_WIDTH)), ("b4", (MLP_OUT,))]
    out, off = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out


def mlp_features(nodes, normals, kv, direction, centre, scale: float, kmax: float) -> np.ndarray:
    x = np.ascontiguousarray(nodes, np.float64)
    nu = np.ascontiguousarray(normals, np.float64)
    kv = np.ascontiguousarray(np.atleast_1d(kv), np.float64)
    d = np.ascontiguousarray(direction, np.float64)
    c = np.ascontiguousarray(centre, np.float64)
    N, nk = x.shape[0], kv.shape[0]
    phi = np.zeros((nk, N, MLP_IN))
    _check(_load().or_mlp_features(_p(x), _p(nu), N, _p(kv), nk, _p(d), _p(c), float(scale), float(kmax),
                                   _p(phi)), "mlp_features")
    return phi


def mlp_forward(theta, X) -> np.ndarray:
    theta = np.ascontiguousarray(theta, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, MLP_IN)
    Y = np.zeros((X.shape[0], MLP_OUT))
    _check(_load().or_mlp_forward(_p(theta), _p(X), X.shape[0], _p(Y)), "mlp_forward")
    return Y


def mlp_loss(theta, X, T) -> float:
    theta = np.ascontiguousarray(theta, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, MLP_IN)
    T = np.ascontiguousarray(T, np.float64).reshape(-1, MLP_OUT)
    L = np.zeros(1)
    _check(_load().or_mlp_loss(_p(theta), _p(X), _p(T), X.shape[0], _p(L)), "mlp_loss")
    return float(L[0])


def mlp_loss_grad(theta, X, T):
    theta = np.ascontiguousarray(theta, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, MLP_IN)
    T = np.ascontiguousarray(T, np.float64).reshape(-1, MLP_OUT)
    L = np.zeros(1)
    g = np.zeros(theta.shape[0])
    _check(_load().or_mlp_loss_grad(_p(theta), _p(X), _p(T), X.shape[0], _p(L), _p(g)), "mlp_loss_grad")
    return float(L[0]), g


def adam_step(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """In place on theta, m, v (float64 arrays)."""
    for a in (theta, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(_load().or_adam_step(theta.shape[0], _p(theta), _p(grad), _p(m), _p(v), int(t), float(lr),
                                float(beta1), float(beta2), float(eps)), "adam_step")
