"""FP64 CPU oracle for planewave-orbital splines (arXiv:1309.6250).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  The product path (the CUDA
library and its Python binding) never imports, links or calls anything here, and the
two share no code: the only thing both sides consume is the seeded input generator.

What the oracle computes, in the paper's order:

1. Grid values of a planewave orbital, Eq. (pw_orbital) sampled at the grid points
   s = l/N: the coefficients are folded onto the N-periodic frequency grid and summed
   with an inverse FFT (a library step; numpy.fft).  `direct_grid_sum` is the same sum
   written out term by term for small cases and for sampled grid points.
2. Spline coefficients (Appendix "B-splines"):
   * interpolating: three stages of cyclic tridiagonal solves with the rows
     [b(1), b(0), b(1)] = [1/4, 1, 1/4] of Eq. (bsplinegridcenteredbasis), solved by
     the Thomas algorithm with a Sherman-Morrison correction for the corners;
   * smoothing: Eq. (b-splinecoefficients), beta = sum_G c_G/gamma_G exp(iG.x);
   * separate Laplacian table (Sec. III A, III C): the same with -|G|^2 c_G.
3. Lagrange tables (Appendix "Lagrange interpolation", Sec. III C): grid values of
   phi, d_x phi, d_y phi, d_z phi and lap phi.
4. pp-spline tables (Appendix "Piecewise-polynomial-form splines"): periodic
   [4 1 ... 1] solves with right-hand side 6 x second differences, applied along each
   axis of the coefficient's label, Eq. (pp-splinecoefficients3).
5. Evaluation and adjoint: plain C loops in qmcspl_oracle.c.
6. Bloch orbitals at k != 0 (Sec. II): tables of the complex periodic part u_nk as
   interleaved real and imaginary functions, evaluated by the same C loops, then
   multiplied by exp(i k.r) with the product rule (bloch_combine).
7. A consumer of the outputs (Sec. I): Slater matrices per walker and spin block, the
   log-determinant, the local kinetic energy and the drift (slater_kinetic).
8. Interpolating B-splines of any odd degree on uniform or non-uniform periodic grids: the
   Appendix's recurrence for the basis, dense periodic interpolation matrices, brute-force
   evaluation and its transpose (general_interp_tables, general_eval, general_adjoint).

Readings of the paper that the code depends on:
* gamma_G (Eq. b-splinecoefficients) is a product over axes of
  3(3 - 4 cos th + cos 2 th)/th^4 with th = 2 pi n_m / N_m the phase per grid step;
  that equals 24 sin^4(th/2)/th^4 = (3/2) sinc^4(th/2) per axis and 3/2 at th = 0.
  The second and third printed forms put the constant outside the product; they are
  read as misprints.
* The pp right-hand side 6/h^2 is taken with h = 1 (reduced units).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmcspl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GCC_FLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile qmcspl_oracle.c into liboracle.so (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", *GCC_FLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L = ctypes.c_long
            I = ctypes.c_int
            lib.orc_bspline_eval.argtypes = [dp, dp, ip, I, dp, L, dp, dp, dp, dp]
            lib.orc_bspline_reduced_derivative.argtypes = [dp, ip, I, dp, L, dp, I, I, I, dp]
            lib.orc_lagrange_eval.argtypes = [dp, ip, I, dp, L, dp, dp, dp, dp]
            lib.orc_lagrange_reduced_derivative.argtypes = [dp, ip, I, dp, L, dp, I, I, I, dp]
            lib.orc_pp_eval.argtypes = [dp, ip, I, dp, L, dp, dp, dp, dp]
            lib.orc_pw_eval.argtypes = [I, ip, I, dp, dp, L, dp, dp, dp, dp, dp]
            lib.orc_bspline_adjoint.argtypes = [dp, dp, ip, I, dp, L, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_set_threads.argtypes = [I]
            lib.orc_set_threads.restype = None
            lib.orc_get_threads.argtypes = []
            lib.orc_get_threads.restype = I
            for name in ("orc_bspline_basis", "orc_lagrange_basis", "orc_pp_basis"):
                getattr(lib, name).argtypes = [ctypes.c_double, I, dp]
                getattr(lib, name).restype = None
            _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads of the C loops (timing only); returns the previous count."""
    lib = _load()
    prev = lib.orc_get_threads()
    lib.orc_set_threads(int(n))
    return prev


def _d(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------------------
# basis polynomials (for pins)
# ---------------------------------------------------------------------------

def basis(kind: str, t: float, d: int = 0) -> np.ndarray:
    """Basis weights at reduced coordinate t: kind in {bspline, lagrange, pp}."""
    lib = _load()
    w = np.zeros(4)
    fn = {"bspline": lib.orc_bspline_basis, "lagrange": lib.orc_lagrange_basis,
          "pp": lib.orc_pp_basis}[kind]
    fn(float(t), int(d), _d(w))
    return w


# ---------------------------------------------------------------------------
# planewave side, Eq. (pw_orbital)
# ---------------------------------------------------------------------------

def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Matrix whose columns are the reciprocal vectors b_i = 2 pi (a^-T)_i."""
    return 2.0 * np.pi * np.linalg.inv(_f64(lattice)).T


def g_vectors(lattice: np.ndarray, miller: np.ndarray) -> np.ndarray:
    """Cartesian G = 2 pi a^-T n for every Miller triple, [n_pw, 3]."""
    return miller.astype(np.float64) @ reciprocal(lattice).T


def pw_eval(lattice, miller, coef, pos) -> Tuple[np.ndarray, np.ndarray, np.ndarray, float]:
    """Direct planewave sums: (val [P,O], grad [P,3,O], lap [P,O], max |Im val|)."""
    lib = _load()
    miller = np.ascontiguousarray(miller, dtype=np.int32)
    coef = np.ascontiguousarray(coef, dtype=np.complex128)
    n_orb, n_pw = coef.shape
    c2 = np.ascontiguousarray(coef.view(np.float64).reshape(n_orb, n_pw, 2))
    pos = _f64(pos).reshape(-1, 3)
    P = pos.shape[0]
    val = np.zeros((P, n_orb))
    grad = np.zeros((P, 3, n_orb))
    lap = np.zeros((P, n_orb))
    mi = np.zeros(1)
    rc = lib.orc_pw_eval(n_pw, _i(miller), n_orb, _d(c2), _d(_f64(lattice)), P, _d(pos),
                         _d(val), _d(grad), _d(lap), _d(mi))
    if rc != 0:
        raise RuntimeError("orc_pw_eval failed (%d)" % rc)
    return val, grad, lap, float(mi[0])


def fold(miller: np.ndarray, weighted: np.ndarray, dims) -> np.ndarray:
    """X[o, k1, k2, k3] = sum over G with n = k (mod N) of weighted[o, G]."""
    n_orb = weighted.shape[0]
    X = np.zeros((n_orb,) + tuple(int(d) for d in dims), dtype=np.complex128)
    k = np.mod(miller.astype(np.int64), np.asarray(dims, dtype=np.int64))
    for o in range(n_orb):
        np.add.at(X[o], (k[:, 0], k[:, 1], k[:, 2]), weighted[o])
    return X


def grid_sum(X: np.ndarray) -> Tuple[np.ndarray, float]:
    """f(x_l) = sum_k X_k exp(2 pi i k.l / N) on the grid, canonical [Nx,Ny,Nz,O].

    The inverse FFT computes the sum divided by N1 N2 N3; it is multiplied back.
    Returns the real part and the largest |imaginary part| (zero for Hermitian input).
    """
    n = X.shape[1] * X.shape[2] * X.shape[3]
    f = np.fft.ifftn(X, axes=(1, 2, 3)) * n
    im = float(np.max(np.abs(f.imag))) if f.size else 0.0
    return np.ascontiguousarray(np.moveaxis(f.real, 0, -1)), im


def direct_grid_sum(miller: np.ndarray, weighted: np.ndarray, dims, points: np.ndarray) -> np.ndarray:
    """The same sum written out: f[l, o] = sum_G weighted[o,G] exp(2 pi i n.l/N).

    `points` are integer grid indices [M, 3].  Returns the real part [M, O].
    """
    frac = points.astype(np.float64) / np.asarray(dims, dtype=np.float64)
    ph = 2.0 * np.pi * (frac @ miller.astype(np.float64).T)     # [M, n_pw]
    return np.real(np.exp(1j * ph) @ weighted.T)


def grid_values(lattice, miller, coef, dims, what: str = "value") -> np.ndarray:
    """Grid values [Nx,Ny,Nz,O] of phi_PW or one of its derivatives.

    what: 'value', 'dx', 'dy', 'dz' (Cartesian derivative) or 'lap'.
    """
    G = g_vectors(lattice, miller)
    if what == "value":
        w = coef
    elif what in ("dx", "dy", "dz"):
        a = "xyz".index(what[1])
        w = coef * (1j * G[:, a])[None, :]
    elif what == "lap":
        w = coef * (-np.einsum("ij,ij->i", G, G))[None, :]
    else:
        raise ValueError(what)
    f, _ = grid_sum(fold(miller, w, dims))
    return f


# ---------------------------------------------------------------------------
# smoothing B-spline, Eq. (b-splinecoefficients)
# ---------------------------------------------------------------------------

def gamma_axis(theta: np.ndarray) -> np.ndarray:
    """One axis of gamma_G: 3(3 - 4 cos th + cos 2th)/th^4, written as 24 sin^4(th/2)/th^4
    (the same function; this form has no cancellation at small th), 3/2 at th = 0."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.full(theta.shape, 1.5)
    nz = theta != 0.0
    th = theta[nz]
    out[nz] = 24.0 * np.sin(0.5 * th) ** 4 / th ** 4
    return out


def gamma(miller: np.ndarray, dims) -> np.ndarray:
    """gamma_G for every planewave: product over axes of gamma_axis(2 pi n_m / N_m)."""
    th = 2.0 * np.pi * miller.astype(np.float64) / np.asarray(dims, dtype=np.float64)
    return gamma_axis(th[:, 0]) * gamma_axis(th[:, 1]) * gamma_axis(th[:, 2])


def smoothing_coefficients(lattice, miller, coef, dims, laplacian: bool = False) -> np.ndarray:
    """beta [Nx,Ny,Nz,O] = sum_G c_G / gamma_G exp(i G.x_lmn); with laplacian=True the
    coefficients of the separate Laplacian spline (c_G -> -|G|^2 c_G)."""
    w = coef / gamma(miller, dims)[None, :]
    if laplacian:
        G = g_vectors(lattice, miller)
        w = w * (-np.einsum("ij,ij->i", G, G))[None, :]
    f, _ = grid_sum(fold(miller, w, dims))
    return f


def smoothing_coefficients_at(lattice, miller, coef, dims, points, laplacian: bool = False):
    """Eq. (b-splinecoefficients) summed directly at selected grid points [M,3] -> [M,O]."""
    w = coef / gamma(miller, dims)[None, :]
    if laplacian:
        G = g_vectors(lattice, miller)
        w = w * (-np.einsum("ij,ij->i", G, G))[None, :]
    return direct_grid_sum(miller, w, dims, points)


# ---------------------------------------------------------------------------
# interpolating B-spline: three stages of cyclic tridiagonal solves
# ---------------------------------------------------------------------------

def cyclic_tridiagonal_solve(rhs: np.ndarray, axis: int, diag: float, off: float) -> np.ndarray:
    """Solve off*x[i-1] + diag*x[i] + off*x[i+1] = rhs[i] (indices mod n) along `axis`.

    Thomas algorithm on the tridiagonal part with a Sherman-Morrison rank-one
    correction for the two corner entries, vectorised over all other axes.
    """
    r = np.moveaxis(np.asarray(rhs, dtype=np.float64), axis, 0)
    n = r.shape[0]
    if n < 3:
        raise ValueError("cyclic solve needs at least 3 points")
    gam = -diag
    dmod = np.full(n, diag)
    dmod[0] = diag - gam
    dmod[-1] = diag - off * off / gam

    def thomas(d):
        cp = np.empty(n)
        dp = np.empty_like(d)
        cp[0] = off / dmod[0]
        dp[0] = d[0] / dmod[0]
        for i in range(1, n):
            m = dmod[i] - off * cp[i - 1]
            cp[i] = off / m
            dp[i] = (d[i] - off * dp[i - 1]) / m
        x = np.empty_like(d)
        x[-1] = dp[-1]
        for i in range(n - 2, -1, -1):
            x[i] = dp[i] - cp[i] * x[i + 1]
        return x

    y = thomas(r)
    u = np.zeros(n)
    u[0] = gam
    u[-1] = off
    q = thomas(u)
    # v = (1, 0, ..., 0, off/gam)
    vy = y[0] + (off / gam) * y[-1]
    vq = q[0] + (off / gam) * q[-1]
    x = y - (vy / (1.0 + vq)) * q.reshape((n,) + (1,) * (y.ndim - 1))
    return np.moveaxis(x, 0, axis)


def interpolating_coefficients(values: np.ndarray) -> np.ndarray:
    """beta with sum_lmn B^x_il B^y_jm B^z_kn beta_lmn = values_ijk (Appendix, interpolating
    B-spline coefficients), solved in three stages along x, y and z."""
    b0, b1 = 1.0, 0.25      # b(0) and b(+-1) of Eq. (bsplinegridcenteredbasis)
    beta = np.asarray(values, dtype=np.float64)
    for axis in range(3):
        beta = cyclic_tridiagonal_solve(beta, axis, b0, b1)
    return np.ascontiguousarray(beta)


def interpolating_tables(lattice, miller, coef, dims, laplacian: bool = False):
    """(beta, beta_lap or None) of the interpolating B-spline."""
    beta = interpolating_coefficients(grid_values(lattice, miller, coef, dims, "value"))
    lap = None
    if laplacian:
        lap = interpolating_coefficients(grid_values(lattice, miller, coef, dims, "lap"))
    return beta, lap


def smoothing_tables(lattice, miller, coef, dims, laplacian: bool = False):
    beta = smoothing_coefficients(lattice, miller, coef, dims)
    lap = smoothing_coefficients(lattice, miller, coef, dims, laplacian=True) if laplacian else None
    return beta, lap


def derivative_tables(method: str, lattice, miller, coef, dims) -> np.ndarray:
    """[5, Nx, Ny, Nz, O]: B-spline coefficients of separate approximations (Sec. III C)
    of phi, d_x phi, d_y phi, d_z phi and lap phi, each built from its own planewave sum
    (multipliers 1, i G_a, -|G|^2): smoothing by Eq. (b-splinecoefficients), interpolating
    by the cyclic solves of the grid values."""
    out = []
    G = g_vectors(lattice, miller)
    for what in ("value", "dx", "dy", "dz", "lap"):
        if method == "smooth":
            if what == "value":
                m = np.ones(G.shape[0], dtype=np.complex128)
            elif what == "lap":
                m = -np.einsum("ij,ij->i", G, G).astype(np.complex128)
            else:
                m = 1j * G[:, "xyz".index(what[1])]
            w = np.asarray(coef) * (m / gamma(miller, dims))[None, :]
            f, _ = grid_sum(fold(miller, w, dims))
            out.append(f)
        elif method == "interp":
            out.append(interpolating_coefficients(grid_values(lattice, miller, coef, dims, what)))
        else:
            raise ValueError(method)
    return np.ascontiguousarray(np.stack(out))


def bspline_eval_separate(tabs, lattice, pos):
    """Value, gradient and Laplacian from five separate B-spline approximations: each is the
    value of its own spline (no derivatives of the value spline, no chain rule)."""
    val = bspline_eval(tabs[0], lattice, pos)[0]
    grad = np.stack([bspline_eval(tabs[1 + a], lattice, pos)[0] for a in range(3)], axis=1)
    lap = bspline_eval(tabs[4], lattice, pos)[0]
    return val, grad, lap


# ---------------------------------------------------------------------------
# Lagrange and pp-spline tables
# ---------------------------------------------------------------------------

def lagrange_tables(lattice, miller, coef, dims) -> np.ndarray:
    """[5, Nx, Ny, Nz, O]: grid values of phi, d_x phi, d_y phi, d_z phi, lap phi."""
    return np.ascontiguousarray(np.stack(
        [grid_values(lattice, miller, coef, dims, w) for w in ("value", "dx", "dy", "dz", "lap")]))


def pp_second_derivative(f: np.ndarray, axis: int) -> np.ndarray:
    """Periodic cubic-spline second derivatives along `axis`:
    [4 1 ... 1; 1 4 1 ...; ...; 1 ... 1 4] sigma = 6/h^2 (f[i-1] - 2 f[i] + f[i+1]), h = 1."""
    rhs = 6.0 * (np.roll(f, 1, axis=axis) - 2.0 * f + np.roll(f, -1, axis=axis))
    return cyclic_tridiagonal_solve(rhs, axis, 4.0, 1.0)


def pp_tables(values: np.ndarray) -> np.ndarray:
    """[8, Nx, Ny, Nz, O] sigma^{kappa mu nu}, index 4(kappa-1) + 2(mu-1) + (nu-1):
    the 1-D operator is applied along every axis whose label is 2."""
    out = []
    for kappa in (1, 2):
        for mu in (1, 2):
            for nu in (1, 2):
                s = np.asarray(values, dtype=np.float64)
                for axis, lab in enumerate((kappa, mu, nu)):
                    if lab == 2:
                        s = pp_second_derivative(s, axis)
                out.append(s)
    return np.ascontiguousarray(np.stack(out))


# ---------------------------------------------------------------------------
# Bloch orbitals at k != 0 (Sec. II): phi_nk(r) = u_nk(r) exp(i k.r)
# ---------------------------------------------------------------------------
# u_nk = sum_G c_G exp(i G.r) is lattice-periodic but complex, so its real and imaginary
# parts are two real functions on the grid (twice the data of a Gamma-point orbital).
# Tables are built for both and stored as adjacent functions (Re u_0, Im u_0, Re u_1, ...);
# the factor exp(i k.r) is applied after the polynomial evaluation, with the
# UNWRAPPED position r.  Separate derivative tables approximate the periodic parts of
# the derivatives of phi itself: grad phi = exp(i k.r) sum_G i(k+G) c_G exp(i G.r) and
# lap phi = -exp(i k.r) sum_G |k+G|^2 c_G exp(i G.r).

def kvector(lattice, kpoint) -> np.ndarray:
    """Cartesian k = 2 pi a^-T kpoint (kpoint in units of the reciprocal vectors)."""
    return reciprocal(lattice) @ np.asarray(kpoint, dtype=np.float64)


def bloch_pw_eval(lattice, miller, coef, kpoint, pos):
    """Direct planewave sums of Bloch orbitals (complex):
    phi = sum_G c_G e^{i(k+G).r}, grad phi = sum_G i(k+G) c_G e^{...}, lap phi = -sum_G |k+G|^2 c_G e^{...}."""
    K = g_vectors(lattice, miller) + kvector(lattice, kpoint)[None, :]      # [n_pw, 3]
    pos = _f64(pos).reshape(-1, 3)
    E = np.exp(1j * (pos @ K.T))                                            # [P, n_pw]
    c = np.asarray(coef, dtype=np.complex128)
    val = E @ c.T
    grad = np.stack([(E * (1j * K[:, a])[None, :]) @ c.T for a in range(3)], axis=1)
    lap = (E * (-np.einsum("ij,ij->i", K, K))[None, :]) @ c.T
    return val, grad, lap


def interleave(z: np.ndarray) -> np.ndarray:
    """Complex [..., O] -> real [..., 2O] with Re and Im of each orbital adjacent."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.empty(z.shape[:-1] + (2 * z.shape[-1],))
    out[..., 0::2] = z.real
    out[..., 1::2] = z.imag
    return out


def deinterleave(x: np.ndarray) -> np.ndarray:
    """Inverse of interleave: real [..., 2O] -> complex [..., O]."""
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0::2] + 1j * x[..., 1::2]


def _complex_grid(miller, weighted, dims) -> np.ndarray:
    """sum_G weighted[o,G] exp(i G.x_l) on the grid, complex [Nx,Ny,Nz,O] (inverse FFT x N)."""
    X = fold(miller, weighted, dims)
    n = X.shape[1] * X.shape[2] * X.shape[3]
    return np.moveaxis(np.fft.ifftn(X, axes=(1, 2, 3)) * n, 0, -1)


def bloch_derivative_weights(lattice, miller, kpoint, what: str) -> np.ndarray:
    """Per-planewave multiplier of the periodic part of phi or a derivative of phi:
    'value' 1, 'dx'/'dy'/'dz' i(k+G)_a, 'lap' -|k+G|^2."""
    K = g_vectors(lattice, miller) + kvector(lattice, kpoint)[None, :]
    if what == "value":
        return np.ones(K.shape[0], dtype=np.complex128)
    if what in ("dx", "dy", "dz"):
        return 1j * K[:, "xyz".index(what[1])]
    if what == "lap":
        return -np.einsum("ij,ij->i", K, K).astype(np.complex128)
    raise ValueError(what)


def bloch_grid_values(lattice, miller, coef, kpoint, dims, what: str = "value") -> np.ndarray:
    """Grid values of the periodic part of phi (u) or of one of its derivatives,
    interleaved real [Nx,Ny,Nz,2O]."""
    w = np.asarray(coef) * bloch_derivative_weights(lattice, miller, kpoint, what)[None, :]
    return interleave(_complex_grid(miller, w, dims))


def bloch_tables(method: str, lattice, miller, coef, kpoint, dims, laplacian: bool = False,
                 gradient: bool = False):
    """Tables of u_nk (and of the periodic part of lap phi) for every method, interleaved.

    smooth: (beta, beta_lap or None), Eq. (b-splinecoefficients) applied to u's coefficients;
    interp: (beta, beta_lap or None), the cyclic systems solved for Re and Im separately;
    lagrange: [5, Nx, Ny, Nz, 2O] grid values of u and of the periodic parts of grad phi, lap phi;
    pp: [8, Nx, Ny, Nz, 2O] pp coefficients of Re u and Im u.
    gradient=True (smooth, interp): [5, Nx, Ny, Nz, 2O] B-spline coefficients of u and of the
    periodic parts of d_x phi, d_y phi, d_z phi and lap phi (separate approximations).
    """
    if gradient and method in ("smooth", "interp"):
        out = []
        for what in ("value", "dx", "dy", "dz", "lap"):
            if method == "smooth":
                w = np.asarray(coef) * (bloch_derivative_weights(lattice, miller, kpoint, what) /
                                        gamma(miller, dims))[None, :]
                out.append(interleave(_complex_grid(miller, w, dims)))
            else:
                out.append(interpolating_coefficients(bloch_grid_values(lattice, miller, coef, kpoint, dims, what)))
        return np.ascontiguousarray(np.stack(out))
    if method == "smooth":
        w = np.asarray(coef) / gamma(miller, dims)[None, :]
        beta = interleave(_complex_grid(miller, w, dims))
        lap = None
        if laplacian:
            wl = w * bloch_derivative_weights(lattice, miller, kpoint, "lap")[None, :]
            lap = interleave(_complex_grid(miller, wl, dims))
        return beta, lap
    if method == "interp":
        beta = interpolating_coefficients(bloch_grid_values(lattice, miller, coef, kpoint, dims))
        lap = None
        if laplacian:
            lap = interpolating_coefficients(bloch_grid_values(lattice, miller, coef, kpoint, dims, "lap"))
        return beta, lap
    if method == "lagrange":
        return np.ascontiguousarray(np.stack(
            [bloch_grid_values(lattice, miller, coef, kpoint, dims, w)
             for w in ("value", "dx", "dy", "dz", "lap")]))
    if method == "pp":
        return pp_tables(bloch_grid_values(lattice, miller, coef, kpoint, dims))
    raise ValueError(method)


def bloch_combine(val, grad, lap, lattice, kpoint, pos, grad_of_u: bool = True, lap_of_u: bool = True):
    """Outputs of phi = u e^{ik.r} from those of the interleaved u tables (real [P,2O], [P,3,2O],
    [P,2O]) -> complex [P,O], [P,3,O], [P,O]:
      phi = e^{ik.r} u
      grad phi = e^{ik.r} (grad u + i k u)               (grad_of_u; else grad is already
                                                          the periodic part of grad phi)
      lap phi = e^{ik.r} (lap u + 2 i k.grad u - |k|^2 u)  (lap_of_u; else lap is already
                                                          the periodic part of lap phi)."""
    k = kvector(lattice, kpoint)
    pos = _f64(pos).reshape(-1, 3)
    ph = np.exp(1j * (pos @ k))[:, None]
    u, gu, lu = deinterleave(val), deinterleave(grad), deinterleave(lap)
    gphi = gu + 1j * k[None, :, None] * u[:, None, :] if grad_of_u else gu
    lphi = lu + 2j * np.einsum("a,pao->po", k, gu) - float(k @ k) * u if lap_of_u else lu
    return ph * u, ph[:, :, None] * gphi, ph * lphi


def bloch_eval(method: str, tables, lattice, kpoint, pos, tables_lap=None):
    """Bloch-orbital value, gradient and Laplacian (complex) through the oracle evaluators
    of each method on interleaved u tables, then bloch_combine."""
    if method in ("smooth", "interp") and np.ndim(tables) == 5:   # separate gradient tables
        v, g, l = bspline_eval_separate(tables, lattice, pos)
        return bloch_combine(v, g, l, lattice, kpoint, pos, False, False)
    if method in ("smooth", "interp"):
        v, g, l = bspline_eval(tables, lattice, pos, beta_lap=tables_lap)
        return bloch_combine(v, g, l, lattice, kpoint, pos, True, tables_lap is None)
    if method == "lagrange":
        v, g, l = lagrange_eval(tables, lattice, pos)
        return bloch_combine(v, g, l, lattice, kpoint, pos, False, False)
    if method == "pp":
        v, g, l = pp_eval(tables, lattice, pos)
        return bloch_combine(v, g, l, lattice, kpoint, pos, True, True)
    raise ValueError(method)


# ---------------------------------------------------------------------------
# evaluation (C loops)
# ---------------------------------------------------------------------------

def _outputs(P, n_orb):
    return np.zeros((P, n_orb)), np.zeros((P, 3, n_orb)), np.zeros((P, n_orb))


def bspline_eval(beta, lattice, pos, beta_lap=None):
    """Tricubic B-spline value, Cartesian gradient and Laplacian, [P,O], [P,3,O], [P,O]."""
    lib = _load()
    beta = _f64(beta)
    dims = _dims(beta.shape[:3])
    n_orb = beta.shape[3]
    pos = _f64(pos).reshape(-1, 3)
    val, grad, lap = _outputs(pos.shape[0], n_orb)
    bl = None if beta_lap is None else _f64(beta_lap)
    rc = lib.orc_bspline_eval(_d(beta), _d(bl), _i(dims), n_orb, _d(_f64(lattice)),
                              pos.shape[0], _d(pos), _d(val), _d(grad), _d(lap))
    if rc:
        raise RuntimeError("orc_bspline_eval failed (%d)" % rc)
    return val, grad, lap


def bspline_reduced_derivative(beta, lattice, pos, order):
    lib = _load()
    beta = _f64(beta)
    dims = _dims(beta.shape[:3])
    n_orb = beta.shape[3]
    pos = _f64(pos).reshape(-1, 3)
    out = np.zeros((pos.shape[0], n_orb))
    rc = lib.orc_bspline_reduced_derivative(_d(beta), _i(dims), n_orb, _d(_f64(lattice)),
                                            pos.shape[0], _d(pos), *[int(x) for x in order], _d(out))
    if rc:
        raise RuntimeError("orc_bspline_reduced_derivative failed")
    return out


def lagrange_eval(tabs, lattice, pos):
    lib = _load()
    tabs = _f64(tabs)
    dims = _dims(tabs.shape[1:4])
    n_orb = tabs.shape[4]
    pos = _f64(pos).reshape(-1, 3)
    val, grad, lap = _outputs(pos.shape[0], n_orb)
    rc = lib.orc_lagrange_eval(_d(tabs), _i(dims), n_orb, _d(_f64(lattice)), pos.shape[0],
                               _d(pos), _d(val), _d(grad), _d(lap))
    if rc:
        raise RuntimeError("orc_lagrange_eval failed")
    return val, grad, lap


def lagrange_reduced_derivative(tab, lattice, pos, order):
    lib = _load()
    tab = _f64(tab)
    dims = _dims(tab.shape[:3])
    n_orb = tab.shape[3]
    pos = _f64(pos).reshape(-1, 3)
    out = np.zeros((pos.shape[0], n_orb))
    rc = lib.orc_lagrange_reduced_derivative(_d(tab), _i(dims), n_orb, _d(_f64(lattice)),
                                             pos.shape[0], _d(pos), *[int(x) for x in order], _d(out))
    if rc:
        raise RuntimeError("orc_lagrange_reduced_derivative failed")
    return out


def pp_eval(sig, lattice, pos):
    lib = _load()
    sig = _f64(sig)
    dims = _dims(sig.shape[1:4])
    n_orb = sig.shape[4]
    pos = _f64(pos).reshape(-1, 3)
    val, grad, lap = _outputs(pos.shape[0], n_orb)
    rc = lib.orc_pp_eval(_d(sig), _i(dims), n_orb, _d(_f64(lattice)), pos.shape[0], _d(pos),
                         _d(val), _d(grad), _d(lap))
    if rc:
        raise RuntimeError("orc_pp_eval failed")
    return val, grad, lap


def bspline_adjoint(beta, lattice, pos, gv, gg, gl, beta_lap=None):
    """(dbeta [Nx,Ny,Nz,O], dbeta_lap or None, dpos [P,3]) for loss = <gv,val>+<gg,grad>+<gl,lap>."""
    lib = _load()
    beta = _f64(beta)
    dims = _dims(beta.shape[:3])
    n_orb = beta.shape[3]
    pos = _f64(pos).reshape(-1, 3)
    P = pos.shape[0]
    dbeta = np.zeros_like(beta)
    bl = None if beta_lap is None else _f64(beta_lap)
    dbl = None if beta_lap is None else np.zeros_like(beta)
    dpos = np.zeros((P, 3))
    rc = lib.orc_bspline_adjoint(_d(beta), _d(bl), _i(dims), n_orb, _d(_f64(lattice)), P, _d(pos),
                                 _d(_f64(gv)), _d(_f64(gg)), _d(_f64(gl)), _d(dbeta), _d(dbl),
                                 _d(dpos))
    if rc:
        raise RuntimeError("orc_bspline_adjoint failed")
    return dbeta, dbl, dpos


# ---------------------------------------------------------------------------
# interpolating B-splines of any odd degree on uniform or non-uniform periodic grids
# (Sec. II "Common features" and "Grid"; Appendix, the B-spline recurrence)
# ---------------------------------------------------------------------------
# The recurrence of the Appendix: b_j^0 = C on [x_j, x_{j+1}), and
#     b_j^k(x) = w_j^k(x) b_j^{k-1}(x) + (1 - w_{j+1}^k(x)) b_{j+1}^{k-1}(x),
#     w_j^k(x) = (x - x_j) / (x_{j+k} - x_j),
# so b_j^k lives on (x_j, x_{j+k+1}); the basis function of grid point m is b_j^k with
# j = m - floor((k+1)/2) (centred on x_m for odd k).  The knots of a periodic axis are the
# grid points x_0 < ... < x_{N-1} in [0, 1) extended by x_{j+N} = x_j + 1.  C is the degree-0
# constant; the paper takes C = 3/2 so that the cubic basis peaks at one, and for degree n
# the same rule gives C_n = 1 / B_n(0) with B_n the unit-sum centred B-spline on unit spacing.

def periodic_knot(knots: np.ndarray, j):
    """x_j of the periodic extension of the grid points knots[0..N-1] in [0, 1)."""
    j = np.asarray(j)
    n = knots.shape[0]
    return knots[np.mod(j, n)] + np.floor_divide(j, n)


def recurrence_basis(knots: np.ndarray, k: int, j, x: float, C: float):
    """b_j^k(x) for an array of start indices j, by the recurrence written out level by level."""
    j = np.asarray(j)
    # level 0 on the start indices j, j+1, ..., j+k (all that level k needs)
    js = j[..., None] + np.arange(k + 1)
    b = np.where((periodic_knot(knots, js) <= x) & (x < periodic_knot(knots, js + 1)), C, 0.0)
    for kk in range(1, k + 1):
        jj = js[..., : k + 1 - kk]
        xj, xjk = periodic_knot(knots, jj), periodic_knot(knots, jj + kk)
        xj1, xj1k = periodic_knot(knots, jj + 1), periodic_knot(knots, jj + 1 + kk)
        w = (x - xj) / (xjk - xj)
        w1 = (x - xj1) / (xj1k - xj1)
        b = w * b[..., :-1] + (1.0 - w1) * b[..., 1:]
    return b[..., 0]


def recurrence_basis_derivative(knots: np.ndarray, k: int, j, x: float, C: float, order: int):
    """d^order/dx^order b_j^k(x): d/dx b_j^k = k (b_j^{k-1}/(x_{j+k}-x_j) - b_{j+1}^{k-1}/(x_{j+k+1}-x_{j+1}))."""
    if order == 0:
        return recurrence_basis(knots, k, j, x, C)
    j = np.asarray(j)
    if order > k:        # piecewise constant after k derivatives: zero between knots
        return np.zeros(j.shape)
    a = k / (periodic_knot(knots, j + k) - periodic_knot(knots, j))
    b = k / (periodic_knot(knots, j + k + 1) - periodic_knot(knots, j + 1))
    return (a * recurrence_basis_derivative(knots, k - 1, j, x, C, order - 1) -
            b * recurrence_basis_derivative(knots, k - 1, j + 1, x, C, order - 1))


def degree_constant(degree: int) -> float:
    """C_n = 1 / B_n(0): the degree-0 constant that makes the centred basis peak at one."""
    n = 64
    pts = np.arange(n) / n           # a uniform periodic axis; the recurrence is scale free
    j0 = -((degree + 1) // 2)        # the basis of grid point 0, evaluated at its centre
    return 1.0 / float(recurrence_basis(pts, degree, np.array([j0]), 0.0, 1.0)[0])


def gamma_degree_axis(theta, degree: int) -> np.ndarray:
    """Fourier transform of the centred degree-n basis (degree-0 constant C_n): the unit
    B-spline is the (n+1)-fold convolution of the unit box, so its transform is
    sinc^{n+1}(th/2); times C_n, and C_n at th = 0.  For n = 3 this is the paper's gamma."""
    theta = np.asarray(theta, dtype=np.float64)
    C = 1.5 if degree == 3 else degree_constant(degree)
    out = np.full(theta.shape, C)
    nz = theta != 0.0
    h = 0.5 * theta[nz]
    out[nz] = C * (np.sin(h) / h) ** (degree + 1)
    return out


def smoothing_tables_degree(lattice, miller, coef, dims, degree: int, laplacian: bool = False):
    """Eq. (b-splinecoefficients) for the degree-n basis: beta = sum_G c_G / gamma_G exp(iG.x)
    with gamma_G the product over axes of gamma_degree_axis(2 pi n_m / N_m)."""
    th = 2.0 * np.pi * miller.astype(np.float64) / np.asarray(dims, dtype=np.float64)
    g = gamma_degree_axis(th[:, 0], degree) * gamma_degree_axis(th[:, 1], degree) * \
        gamma_degree_axis(th[:, 2], degree)
    w = np.asarray(coef) / g[None, :]
    beta, _ = grid_sum(fold(miller, w, dims))
    lap = None
    if laplacian:
        G = g_vectors(lattice, miller)
        lap, _ = grid_sum(fold(miller, w * (-np.einsum("ij,ij->i", G, G))[None, :], dims))
    return beta, lap


def axis_points(n: int, knots=None) -> np.ndarray:
    """Grid points of one periodic axis in reduced coordinates: l/N, or the given knots."""
    return np.arange(n) / n if knots is None else np.asarray(knots, dtype=np.float64)


def periodic_basis_matrix(points: np.ndarray, degree: int, x: np.ndarray, C: float, order: int = 0):
    """M[p][m] = sum over periodic images of (d/dx)^order of the basis of grid point m at x[p]."""
    n = points.shape[0]
    M = np.zeros((x.shape[0], n))
    half = (degree + 1) // 2
    j = np.arange(n)[None, :] + n * np.array([-1, 0, 1])[:, None] - half      # [image, m]
    for p, xv in enumerate(x):
        M[p] = recurrence_basis_derivative(points, degree, j, xv, C, order).sum(axis=0)
    return M


def general_grid_values(lattice, miller, coef, points, what: str = "value", kpoint=None):
    """Planewave sum (or its Laplacian, or the periodic part u of a Bloch orbital) at the
    tensor grid of per-axis points, separable: [N1, N2, N3, O] real, or interleaved for kpoint."""
    c = np.asarray(coef, dtype=np.complex128)
    if what == "lap":
        if kpoint is None:
            G = g_vectors(lattice, miller)
            c = c * (-np.einsum("ij,ij->i", G, G))[None, :]
        else:
            c = c * bloch_derivative_weights(lattice, miller, kpoint, "lap")[None, :]
    E = [np.exp(2j * np.pi * np.outer(points[a], miller[:, a].astype(np.float64))) for a in range(3)]
    f = np.einsum("ag,bg,cg,og->abco", E[0], E[1], E[2], c)
    return interleave(f) if kpoint is not None else np.ascontiguousarray(f.real)


def general_interp_tables(lattice, miller, coef, dims, degree: int = 3, knots=(None, None, None),
                          laplacian: bool = False, kpoint=None):
    """(beta, beta_lap or None): sum_lmn B^x_il B^y_jm B^z_kn beta_lmn = phi(x_i, y_j, z_k) with the
    basis of the recurrence (C = 3/2 for cubic, C_n otherwise), solved in three stages with dense
    periodic matrices (numpy.linalg.solve as the library step)."""
    C = 1.5 if degree == 3 else degree_constant(degree)
    pts = [axis_points(int(dims[a]), knots[a]) for a in range(3)]
    mats = [periodic_basis_matrix(pts[a], degree, pts[a], C) for a in range(3)]

    def solve(values):
        beta = np.asarray(values, dtype=np.float64)
        for a in range(3):
            beta = np.moveaxis(np.tensordot(np.linalg.inv(mats[a]), np.moveaxis(beta, a, 0), axes=1), 0, a)
        return np.ascontiguousarray(beta)

    beta = solve(general_grid_values(lattice, miller, coef, pts, "value", kpoint))
    lap = solve(general_grid_values(lattice, miller, coef, pts, "lap", kpoint)) if laplacian else None
    return beta, lap


def general_eval(beta, lattice, pos, degree: int = 3, knots=(None, None, None), beta_lap=None):
    """Value, Cartesian gradient, Laplacian of the spline sum_lmn b_l(x) b_m(y) b_n(z) beta_lmn,
    every basis function of the periodic family evaluated by the recurrence (brute force)."""
    beta = np.asarray(beta, dtype=np.float64)
    dims = beta.shape[:3]
    C = 1.5 if degree == 3 else degree_constant(degree)
    pts = [axis_points(int(dims[a]), knots[a]) for a in range(3)]
    ainv = np.linalg.inv(np.asarray(lattice, dtype=np.float64))
    pos = _f64(pos).reshape(-1, 3)
    s = pos @ ainv.T
    s = s - np.floor(s)
    P, O = pos.shape[0], beta.shape[3]
    val, grad, lap = np.zeros((P, O)), np.zeros((P, 3, O)), np.zeros((P, O))
    metric = ainv @ ainv.T                         # (a^-1 a^-T)_ij
    for p in range(P):
        B = [[periodic_basis_matrix(pts[a], degree, s[p, a:a + 1], C, d)[0] for d in range(3)]
             for a in range(3)]
        def tp(dx, dy, dz, tab=beta):
            return np.einsum("l,m,n,lmno->o", B[0][dx], B[1][dy], B[2][dz], tab)
        val[p] = tp(0, 0, 0)
        ds = np.stack([tp(1, 0, 0), tp(0, 1, 0), tp(0, 0, 1)])          # d/ds_i
        grad[p] = ainv.T @ ds
        if beta_lap is not None:
            lap[p] = tp(0, 0, 0, np.asarray(beta_lap, dtype=np.float64))
        else:
            H = np.zeros((3, 3, O))
            for i in range(3):
                for j in range(3):
                    o = [0, 0, 0]
                    o[i] += 1
                    o[j] += 1
                    H[i, j] = tp(*o)
            lap[p] = np.einsum("ij,ijo->o", metric, H)
    return val, grad, lap


def general_adjoint(beta, lattice, pos, gv, gg, gl, degree: int = 3, knots=(None, None, None), beta_lap=None):
    """(dbeta, dbeta_lap or None, dpos [P, 3]) for loss = <gv,val> + <gg,grad> + <gl,lap> with
    the outputs of general_eval: its exact transpose, brute force over every basis function.

    With D_i = d/ds_i and the Cartesian gradient grad = a^-T (D_1, D_2, D_3) phi, the loss
    is linear in beta: each coefficient gets
        gv B + sum_i gt_i D_i B + gl sum_ij M_ij D_i D_j B     (gt = a^-1 gg, M = a^-1 a^-T),
    the last term moving to dbeta_lap (gl B) with a separate Laplacian table.  The position
    adjoint is dL/dr = a^-T u with u_i = sum_o [gv D_i phi + sum_j (D_i D_j phi) gt_j + gl D_i lap],
    D_i lap = sum_jk M_jk D_i D_j D_k phi, or D_i of the Laplacian table."""
    beta = np.asarray(beta, dtype=np.float64)
    dims = beta.shape[:3]
    C = 1.5 if degree == 3 else degree_constant(degree)
    pts = [axis_points(int(dims[a]), knots[a]) for a in range(3)]
    ainv = np.linalg.inv(np.asarray(lattice, dtype=np.float64))
    metric = ainv @ ainv.T
    pos = _f64(pos).reshape(-1, 3)
    s = pos @ ainv.T
    s = s - np.floor(s)
    P = pos.shape[0]
    bl = None if beta_lap is None else np.asarray(beta_lap, dtype=np.float64)
    gv = np.asarray(gv, dtype=np.float64).reshape(P, -1)
    gg = np.asarray(gg, dtype=np.float64).reshape(P, 3, -1)
    gl = np.asarray(gl, dtype=np.float64).reshape(P, -1)
    dbeta = np.zeros_like(beta)
    dbl = None if bl is None else np.zeros_like(beta)
    dpos = np.zeros((P, 3))
    for p in range(P):
        B = [[periodic_basis_matrix(pts[a], degree, s[p, a:a + 1], C, d)[0] for d in range(4)]
             for a in range(3)]

        def basis(o):   # the tensor D_x^o0 D_y^o1 D_z^o2 of every basis function [N1, N2, N3]
            return np.einsum("l,m,n->lmn", B[0][o[0]], B[1][o[1]], B[2][o[2]])

        def unit(*axes):
            o = [0, 0, 0]
            for a in axes:
                o[a] += 1
            return o

        gt = ainv @ gg[p]                                    # [3, O]
        # coefficient adjoint
        dbeta += np.einsum("lmn,o->lmno", basis((0, 0, 0)), gv[p])
        for i in range(3):
            dbeta += np.einsum("lmn,o->lmno", basis(unit(i)), gt[i])
        if bl is None:
            lapB = sum(metric[i, j] * basis(unit(i, j)) for i in range(3) for j in range(3))
            dbeta += np.einsum("lmn,o->lmno", lapB, gl[p])
        else:
            dbl += np.einsum("lmn,o->lmno", basis((0, 0, 0)), gl[p])
        # position adjoint
        val = lambda o, tab=beta: np.einsum("lmn,lmno->o", basis(o), tab)
        u = np.zeros(3)
        for i in range(3):
            ui = gv[p] * val(unit(i))
            for j in range(3):
                ui = ui + val(unit(i, j)) * gt[j]
            if bl is None:
                dlap = sum(metric[j, k] * val(unit(i, j, k)) for j in range(3) for k in range(3))
            else:
                dlap = val(unit(i), bl)
            u[i] = np.sum(ui + gl[p] * dlap)
        dpos[p] = ainv.T @ u
    return dbeta, dbl, dpos


# ---------------------------------------------------------------------------
# Slater-determinant consumer of the orbital outputs (Sec. I)
# ---------------------------------------------------------------------------
# The trial wave function of Sec. I is Psi = J D with D a Slater determinant of the
# single-particle orbitals; without the Jastrow factor and with the electrons split into
# spin blocks, Psi = det A_up det A_dn, A_s[i][j] = phi_j(r_i) over the block's electrons i
# and its first n_s orbitals j.  The kinetic part of the local energy E_L = H Psi / Psi is
# T_L = -1/2 sum_i lap_i Psi / Psi, and by Jacobi's formula (row i of A replaced by its
# Laplacian) lap_i det A / det A = sum_j (A^-1)_ji lap phi_j(r_i), so
# T_L = -1/2 sum_s tr(A_s^-1 L_s) with L_s[i][j] = lap phi_j(r_i); likewise the drift
# grad_i ln|Psi| = sum_j (A^-1)_ji grad phi_j(r_i).

def slater_kinetic(val, grad, lap, n_walkers: int, n_elec: int, n_up: int):
    """Per walker: (logdet [W] = ln|det A_up| + ln|det A_dn|, sign [W], kinetic [W] = T_L,
    drift [W, n_elec, 3]) from orbital outputs val [W*n_elec, O], grad [W*n_elec, 3, O],
    lap [W*n_elec, O] (walker-major positions; electrons 0..n_up-1 spin up).  numpy's
    slogdet and inv serve as library steps.  Complex orbitals (Bloch functions, Sec. II)
    give complex determinants: then sign is the unit complex number det / |det| of the
    product, and the kinetic term and the drift are complex (Jacobi's formula holds as is)."""
    cplx = any(np.iscomplexobj(x) for x in (val, grad, lap))
    dt = np.complex128 if cplx else np.float64
    val = np.asarray(val, dtype=dt)
    grad = np.asarray(grad, dtype=dt)
    lap = np.asarray(lap, dtype=dt)
    logdet = np.zeros(n_walkers)
    sign = np.ones(n_walkers, dtype=dt)
    kin = np.zeros(n_walkers, dtype=dt)
    drift = np.zeros((n_walkers, n_elec, 3), dtype=dt)
    for w in range(n_walkers):
        for e0, n in ((0, n_up), (n_up, n_elec - n_up)):
            if n == 0:
                continue
            rows = slice(w * n_elec + e0, w * n_elec + e0 + n)
            A = val[rows, :n]
            sg, ld = np.linalg.slogdet(A)
            logdet[w] += ld
            sign[w] *= sg
            Ainv = np.linalg.inv(A)
            kin[w] += -0.5 * np.trace(Ainv @ lap[rows, :n])
            drift[w, e0:e0 + n] = np.einsum("ji,iaj->ia", Ainv, grad[rows, :, :n])
    return logdet, sign, kin, drift


# ---------------------------------------------------------------------------
# reduced-precision storage of a table (the benchmark spec's precision pattern: FP64 construction,
# FP32 / BF16 storage)
# ---------------------------------------------------------------------------

def round_to_storage(table: Optional[np.ndarray], storage: str) -> Optional[np.ndarray]:
    """A table of FP64 coefficients as stored in `storage`, back in float64: each value rounded
    once to the nearest representable number, ties to even -- FP32 (24 significant bits) or
    BF16 (8 significant bits, FP32's exponent range); FP64 and double-float ('df64': a float pair
    that carries the FP64 value to about 2^-48) as they are.  Written from the definition of the
    two formats: frexp gives x = m 2^e with 1/2 <= |m| < 1, and m 2^b is rounded to an integer
    (numpy.round is round-half-to-even) for b significant bits.  Values here are far from the
    formats' overflow and subnormal ranges."""
    if table is None or storage in ("f64", "df64"):
        return table
    bits = {"f32": 24, "bf16": 8}[storage]
    x = np.asarray(table, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(np.ldexp(m, bits)), e - bits)


# ---------------------------------------------------------------------------
# error metrics
# ---------------------------------------------------------------------------

def relative_error(test: np.ndarray, ref: np.ndarray) -> float:
    """max |test - ref| / max |ref| (per output, relative to its largest magnitude)."""
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(test))) if test.size else 0.0
    t = np.asarray(test)
    if not np.iscomplexobj(t):
        t = t.astype(np.float64)
    return float(np.max(np.abs(t - ref))) / scale


def relative_mean_absolute_error(test: np.ndarray, ref: np.ndarray) -> float:
    """The paper's accuracy metric (Sec. III A): mean |error| / mean |planewave value|."""
    return float(np.mean(np.abs(test - ref)) / np.mean(np.abs(ref)))


def kinetic_energy(val: np.ndarray, lap: np.ndarray) -> np.ndarray:
    """Per-orbital kinetic-energy estimate over the sampled positions:
    T_n = -1/2 sum_p phi_n lap phi_n / sum_p phi_n^2 (Hartree)."""
    return -0.5 * np.sum(val * lap, axis=0) / np.sum(val * val, axis=0)
