"""Pins of the oracle's Bloch-orbital path (k != 0, Sec. II: phi_nk = u_nk exp(i k.r)).

None of these compares the oracle with itself: the checks are closed forms of a single
planewave at grid points, Bloch's theorem, finite differences, the reduction to the
real Gamma-point path, exact reproduction of grid values by interpolating methods and
the convergence rate under refinement.
"""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs

NONORTHO = np.array([[5.0, 1.0, 0.5],
                     [0.0, 6.0, 0.3],
                     [0.0, 0.0, 7.0]])   # columns are a_1, a_2, a_3
KGEN = inputs.KPOINTS["generic"]


def bloch_tabs(method, lat, mil, coef, kp, dims, sep=False):
    t = oracle.bloch_tables(method, lat, mil, coef, kp, dims, laplacian=sep)
    if method in ("smooth", "interp"):
        return t
    return t, None


def evaluate(method, tabs, lat, kp, pos):
    return oracle.bloch_eval(method, tabs[0], lat, kp, pos, tables_lap=tabs[1])


def test_bloch_planewave_sum_closed_form():
    """Sec. II: one planewave c e^{i(k+G).r} has gradient i(k+G) phi and Laplacian
    -|k+G|^2 phi; a lattice translation R multiplies it by e^{ik.R}."""
    mil = np.array([[1, -2, 1]], dtype=np.int32)
    c = 0.3 - 0.7j
    coef = np.array([[c]])
    rng = np.random.default_rng(1)
    pos = rng.uniform(-10, 10, (40, 3))
    v, g, l = oracle.bloch_pw_eval(NONORTHO, mil, coef, KGEN, pos)
    B = 2 * np.pi * np.linalg.inv(NONORTHO).T
    K = B @ (mil[0] + np.array(KGEN))
    ref = c * np.exp(1j * pos @ K)
    np.testing.assert_allclose(v[:, 0], ref, atol=1e-13)
    np.testing.assert_allclose(g[:, :, 0], 1j * K[None, :] * ref[:, None], atol=1e-12)
    np.testing.assert_allclose(l[:, 0], -(K @ K) * ref, atol=1e-11)
    R = NONORTHO @ np.array([2.0, -1.0, 3.0])
    v2, _, _ = oracle.bloch_pw_eval(NONORTHO, mil, coef, KGEN, pos + R)
    np.testing.assert_allclose(v2, v * np.exp(1j * (B @ np.array(KGEN)) @ R), atol=1e-12)


@pytest.mark.parametrize("shift", [(0, 0, 0), (1, -2, 3)])
def test_bloch_smoothing_single_planewave_at_grid_points(shift):
    """Eq. (b-splinecoefficients) for u = c e^{iG.r} at k != 0, evaluated at grid points
    (t = 0, weights [1/4, 1, 1/4, 0], derivative weights [-3/4, 0, 3/4, 0], second
    derivative weights [3/2, -3, 3/2, 0]): per axis u picks up (1 + cos th/2)/gamma(th),
    d/dt (3/2) i sin th/gamma(th), d2/dt2 3 (cos th - 1)/gamma(th); then
    grad phi = e^{ik.r}(grad u + i k u), lap phi = e^{ik.r}(lap u + 2i k.grad u - |k|^2 u),
    and the separate Laplacian table gives -|k+G|^2 e^{ik.r} u.  Positions are shifted by
    a lattice vector so that the phase must use the unwrapped position."""
    dims = np.array([8, 10, 12])
    n = np.array([1, -2, 3])
    mil = n[None, :].astype(np.int32)
    c = 0.6 + 0.25j
    coef = np.array([[c]])
    lat = NONORTHO
    beta, blap = oracle.bloch_tables("smooth", lat, mil, coef, KGEN, tuple(dims), laplacian=True)
    rng = np.random.default_rng(2)
    j = rng.integers(0, dims, size=(25, 3))
    pos = (j / dims) @ lat.T + lat @ np.array(shift, dtype=float)
    v, g, l = oracle.bloch_eval("smooth", beta, lat, KGEN, pos)
    _, _, lsep = oracle.bloch_eval("smooth", beta, lat, KGEN, pos, tables_lap=blap)

    th = 2 * np.pi * n / dims
    gam = oracle.gamma_axis(th)
    S = (1 + 0.5 * np.cos(th)) / gam
    D1 = 1.5j * np.sin(th) / gam
    D2 = 3.0 * (np.cos(th) - 1.0) / gam
    ainv = np.linalg.inv(lat)
    B = 2 * np.pi * ainv.T
    G = B @ n
    k = B @ np.array(KGEN)
    base = c * np.exp(1j * pos @ G)                       # c e^{iG.r} at the grid points
    u = base * np.prod(S)
    du = np.stack([base * D1[a] * np.prod(np.delete(S, a)) for a in range(3)], axis=1)  # d/dt_a
    H = np.zeros((pos.shape[0], 3, 3), dtype=complex)
    for a in range(3):
        for b in range(3):
            if a == b:
                H[:, a, a] = base * D2[a] * np.prod(np.delete(S, a))
            else:
                o = 3 - a - b
                H[:, a, b] = base * D1[a] * D1[b] * S[o]
    M = dims[:, None] * ainv                              # grad_cart = M^T d/dt
    gu = du @ M
    lu = np.einsum("ia,ja,pij->p", M, M, H)
    ph = np.exp(1j * pos @ k)
    np.testing.assert_allclose(v[:, 0], ph * u, atol=1e-12)
    np.testing.assert_allclose(g[:, :, 0], ph[:, None] * (gu + 1j * k[None, :] * u[:, None]), atol=1e-11)
    np.testing.assert_allclose(l[:, 0], ph * (lu + 2j * gu @ k - (k @ k) * u), atol=1e-10)
    np.testing.assert_allclose(lsep[:, 0], -((G + k) @ (G + k)) * ph * u, atol=1e-10)


@pytest.mark.parametrize("method,sep", [("smooth", False), ("smooth", True), ("interp", False),
                                        ("interp", True), ("lagrange", False), ("pp", False)])
def test_bloch_theorem_for_every_method(method, sep):
    """Sec. II: u is lattice-periodic, so every approximation obeys phi(r + R) = e^{ik.R} phi(r)
    (value, gradient and Laplacian)."""
    dims = (8, 9, 10)
    lat, mil, coef = inputs.random_bloch_cell(11, 3, 5.0, 4.0, KGEN, NONORTHO)
    tabs = bloch_tabs(method, lat, mil, coef, KGEN, dims, sep)
    pos = inputs.positions(lat, 30, 7)
    out0 = evaluate(method, tabs, lat, KGEN, pos)
    k = oracle.kvector(lat, KGEN)
    for m in ([1, 0, 0], [0, -2, 1], [3, 1, -4]):
        R = lat @ np.array(m, dtype=float)
        out = evaluate(method, tabs, lat, KGEN, pos + R)
        f = np.exp(1j * k @ R)
        for a, b in zip(out, out0):
            assert oracle.relative_error(a, f * b) < 1e-12


@pytest.mark.parametrize("method", ["smooth", "interp", "pp"])
def test_bloch_derivatives_by_finite_differences(method):
    """The gradient of the combined orbital is the derivative of its value and the
    Laplacian the divergence of its gradient (product rule with e^{ik.r})."""
    dims = (7, 9, 11)
    lat, mil, coef = inputs.random_bloch_cell(12, 2, 4.0, 4.0, KGEN, NONORTHO)
    tabs = bloch_tabs(method, lat, mil, coef, KGEN, dims)
    pos = inputs.positions(lat, 20, 8)
    v, g, l = evaluate(method, tabs, lat, KGEN, pos)
    h = 1e-5
    fd_g = np.zeros_like(g)
    fd_l = np.zeros_like(l)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        vp, gp, _ = evaluate(method, tabs, lat, KGEN, pos + e)
        vm, gm, _ = evaluate(method, tabs, lat, KGEN, pos - e)
        fd_g[:, a] = (vp - vm) / (2 * h)
        fd_l += (gp[:, a] - gm[:, a]) / (2 * h)
    assert oracle.relative_error(g, fd_g) < 1e-8
    assert oracle.relative_error(l, fd_l) < 1e-6


@pytest.mark.parametrize("method", ["smooth", "interp", "lagrange", "pp"])
def test_bloch_at_gamma_reduces_to_the_real_path(method):
    """k = 0 with Hermitian coefficients: Im u vanishes and Re u is the real orbital, so the
    complex outputs equal the Gamma-point path's (Sec. III)."""
    dims = (8, 8, 10)
    lat, mil, coef = inputs.random_cell(13, dims, 3, 5.0, 4.0, NONORTHO)
    kp = (0.0, 0.0, 0.0)
    pos = inputs.positions(lat, 25, 9, -1, 2)
    if method == "smooth":
        beta, blap = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
        ref = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
        tabs = oracle.bloch_tables("smooth", lat, mil, coef, kp, dims, laplacian=True)
    elif method == "interp":
        beta, blap = oracle.interpolating_tables(lat, mil, coef, dims, laplacian=True)
        ref = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
        tabs = oracle.bloch_tables("interp", lat, mil, coef, kp, dims, laplacian=True)
    elif method == "lagrange":
        ref = oracle.lagrange_eval(oracle.lagrange_tables(lat, mil, coef, dims), lat, pos)
        tabs = (oracle.bloch_tables("lagrange", lat, mil, coef, kp, dims), None)
    else:
        ref = oracle.pp_eval(oracle.pp_tables(oracle.grid_values(lat, mil, coef, dims)), lat, pos)
        tabs = (oracle.bloch_tables("pp", lat, mil, coef, kp, dims), None)
    assert np.abs(tabs[0][..., 1::2]).max() < 1e-12 * np.abs(tabs[0]).max()
    out = evaluate(method, tabs, lat, kp, pos)
    for a, b in zip(out, ref):
        assert oracle.relative_error(a.real, b) < 1e-12
        assert np.abs(a.imag).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("method", ["interp", "lagrange", "pp"])
def test_bloch_interpolating_methods_reproduce_grid_values(method):
    """Interpolating B-splines, Lagrange and pp-splines pass through the grid values of u
    (Appendix), so at a grid point the value equals the planewave sum of the Bloch orbital;
    Lagrange's gradient and Laplacian tables hold the periodic parts of grad phi and lap phi,
    so those equal the planewave sums there too."""
    dims = np.array([8, 9, 10])
    lat, mil, coef = inputs.random_bloch_cell(14, 3, 4.0, 4.0, KGEN, NONORTHO)
    tabs = bloch_tabs(method, lat, mil, coef, KGEN, tuple(dims))
    rng = np.random.default_rng(3)
    j = rng.integers(0, dims, size=(20, 3))
    pos = (j / dims) @ lat.T + lat @ np.array([1.0, -1.0, 2.0])
    v, g, l = evaluate(method, tabs, lat, KGEN, pos)
    pv, pg, pl = oracle.bloch_pw_eval(lat, mil, coef, KGEN, pos)
    assert oracle.relative_error(v, pv) < 1e-12
    if method == "lagrange":
        assert oracle.relative_error(g, pg) < 1e-12
        assert oracle.relative_error(l, pl) < 1e-12


def test_bloch_smoothing_converges_at_fourth_order():
    """Sec. III A footnote at k != 0: refining the grid at fixed cutoff converges the value
    and the separate Laplacian as h^4, the gradient as h^3."""
    lat = np.eye(3) * 5.0
    mil = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 1], [0, -1, 0], [1, -1, 0]], dtype=np.int32)
    coef = np.array([[0.4 + 0.2j, 0.1 - 0.3j, 0.3, -0.2j, 0.25 + 0.05j]])
    pos = inputs.positions(lat, 200, 13)
    pv, pg, pl = oracle.bloch_pw_eval(lat, mil, coef, KGEN, pos)
    errs = []
    for n in (8, 16, 32):
        beta, blap = oracle.bloch_tables("smooth", lat, mil, coef, KGEN, (n, n, n), laplacian=True)
        v, g, _ = oracle.bloch_eval("smooth", beta, lat, KGEN, pos)
        _, _, lt = oracle.bloch_eval("smooth", beta, lat, KGEN, pos, tables_lap=blap)
        errs.append([np.abs(v - pv).max(), np.abs(g - pg).max(), np.abs(lt - pl).max()])
    ratio = np.array(errs[1]) / np.array(errs[2])
    assert ratio[0] > 12 and ratio[2] > 12
    assert ratio[1] > 6


def test_bloch_coefficients_are_not_hermitian_and_cutoff_is_centred_on_minus_k():
    """The generator draws k != 0 coefficients independently (no c_{-G} = conj(c_G)) over
    the sphere |k + G|^2/2 <= Ecut."""
    lat = NONORTHO
    mil = inputs.miller_set(lat, 6.0, KGEN)
    B = 2 * np.pi * np.linalg.inv(lat).T
    K = (mil + np.array(KGEN)) @ B.T
    assert np.all(0.5 * np.sum(K * K, axis=1) <= 6.0 * (1 + 1e-14))
    # every Miller triple just outside the kept set is outside the sphere
    kept = {tuple(m) for m in mil.tolist()}
    for m in mil[:50]:
        for d in np.eye(3, dtype=int):
            for s in (1, -1):
                q = tuple(int(x) for x in m + s * d)
                if q not in kept:
                    kq = (np.array(q) + np.array(KGEN)) @ B.T
                    assert 0.5 * kq @ kq > 6.0
    coef = inputs.bloch_coefficients(lat, mil, 2, KGEN, 4.0, 5)
    v, _, _ = oracle.bloch_pw_eval(lat, mil, coef, KGEN, inputs.positions(lat, 10, 1))
    assert np.abs(v.imag).max() > 1e-3


@pytest.mark.parametrize("method", ["smooth", "interp"])
def test_bloch_separate_gradient_tables(method):
    """Separate gradient tables of a Bloch orbital approximate the periodic part of grad phi,
    sum_G i(k+G) c_G e^{iG.r}: the interpolating ones reproduce the planewave gradient at
    grid points; both obey Bloch's theorem."""
    dims = np.array([8, 9, 10])
    lat, mil, coef = inputs.random_bloch_cell(15, 2, 4.0, 4.0, KGEN, NONORTHO)
    tabs = oracle.bloch_tables(method, lat, mil, coef, KGEN, tuple(dims), gradient=True)
    assert tabs.shape == (5,) + tuple(dims) + (4,)
    rng = np.random.default_rng(4)
    pos = (rng.integers(0, dims, size=(20, 3)) / dims) @ lat.T + lat @ np.array([1.0, 2.0, -1.0])
    v, g, l = oracle.bloch_eval(method, tabs, lat, KGEN, pos)
    if method == "interp":
        pv, pg, pl = oracle.bloch_pw_eval(lat, mil, coef, KGEN, pos)
        for a, b in ((v, pv), (g, pg), (l, pl)):
            assert oracle.relative_error(a, b) < 1e-12
    R = lat @ np.array([2.0, -1.0, 1.0])
    v2, g2, l2 = oracle.bloch_eval(method, tabs, lat, KGEN, pos + R)
    f = np.exp(1j * oracle.kvector(lat, KGEN) @ R)
    for a, b in ((v2, v), (g2, g), (l2, l)):
        assert oracle.relative_error(a, f * b) < 1e-12
