"""Pins of the oracle's Slater-determinant consumer (Sec. I: Psi = det A_up det A_dn,
kinetic part of the local energy E_L = H Psi / Psi).

Checks: the closed form for orbitals that are eigenfunctions of the kinetic operator, finite
differences of the determinant for the drift and for the kinetic energy, antisymmetry under
electron exchange and a hand-expanded 2 x 2 determinant."""
import math

import numpy as np
import pytest

import oracle

LAT = np.array([[6.0, 0.5, 0.0],
                [0.0, 6.5, 0.4],
                [0.0, 0.0, 7.0]])


def shell_orbitals(n_orb):
    """Real orbitals cos(G.r), sin(G.r) for distinct G (each an eigenfunction of -1/2 lap
    with eigenvalue |G|^2/2), as Miller triples and Hermitian coefficients."""
    mil, coef = [], []
    rng = np.random.default_rng(5)
    gs = []
    while len(gs) < (n_orb + 1) // 2:
        g = tuple(int(x) for x in rng.integers(-2, 3, 3))
        if g != (0, 0, 0) and g not in gs and tuple(-x for x in g) not in gs:
            gs.append(g)
    for g in gs:
        mil += [g, tuple(-x for x in g)]
    mil = np.array(mil, dtype=np.int32)
    coef = np.zeros((n_orb, mil.shape[0]), dtype=complex)
    for o in range(n_orb):
        k = o // 2
        if o % 2 == 0:      # cos
            coef[o, 2 * k], coef[o, 2 * k + 1] = 0.5, 0.5
        else:               # sin
            coef[o, 2 * k], coef[o, 2 * k + 1] = -0.5j, 0.5j
    return mil, coef


def outputs(mil, coef, pos):
    v, g, l, _ = oracle.pw_eval(LAT, mil, coef, pos)
    return v, g, l


def test_kinetic_energy_of_eigenfunction_determinant_is_the_sum_of_eigenvalues():
    """If lap phi_j = -|G_j|^2 phi_j then L = A diag(-|G_j|^2) and T_L = 1/2 sum_j |G_j|^2
    for every configuration (both spin blocks)."""
    n_up, n_dn = 6, 4
    mil, coef = shell_orbitals(10)          # more orbitals than either block uses
    B = 2 * np.pi * np.linalg.inv(LAT).T
    g2 = np.array([np.sum((B @ mil[2 * (o // 2)]) ** 2) for o in range(10)])
    expect = 0.5 * (g2[:n_up].sum() + g2[:n_dn].sum())
    rng = np.random.default_rng(6)
    W = 5
    pos = rng.uniform(0, 6, (W * (n_up + n_dn), 3))
    v, g, l = outputs(mil, coef, pos)
    _, _, kin, _ = oracle.slater_kinetic(v, g, l, W, n_up + n_dn, n_up)
    np.testing.assert_allclose(kin, expect, rtol=1e-9)


def _logdet(mil, coef, pos, n_elec, n_up):
    v, g, l = outputs(mil, coef, pos)
    return oracle.slater_kinetic(v, g, l, 1, n_elec, n_up)


def test_drift_and_kinetic_by_finite_differences():
    """drift_i = grad_i ln|D| and T_L = -1/2 sum_i lap_i D / D, by central differences of the
    determinant of generic (non-eigenfunction) orbitals."""
    rng = np.random.default_rng(7)
    n_up, n_elec = 4, 7
    mil = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.int32)
    coef = np.zeros((n_up, mil.shape[0]), dtype=complex)
    idx = {tuple(m): i for i, m in enumerate(mil.tolist())}
    for o in range(n_up):
        for i, m in enumerate(mil.tolist()):
            j = idx[tuple(-x for x in m)]
            if i < j:
                z = complex(*rng.standard_normal(2))
                coef[o, i], coef[o, j] = z, np.conj(z)
            elif i == j:
                coef[o, i] = rng.standard_normal()
    pos = rng.uniform(0, 6, (n_elec, 3))
    ld0, s0, kin, drift = _logdet(mil, coef, pos, n_elec, n_up)
    h = 1e-4
    lap_sum = 0.0
    fd = np.zeros((n_elec, 3))
    for i in range(n_elec):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            lp, sp, _, _ = _logdet(mil, coef, pp, n_elec, n_up)
            lm, sm, _, _ = _logdet(mil, coef, pm, n_elec, n_up)
            fd[i, a] = (lp[0] - lm[0]) / (2 * h)
            # D(r+h)/D(r) and D(r-h)/D(r) for the second difference of D itself
            rp = sp[0] * s0[0] * math.exp(lp[0] - ld0[0])
            rm = sm[0] * s0[0] * math.exp(lm[0] - ld0[0])
            lap_sum += (rp - 2.0 + rm) / h ** 2
    np.testing.assert_allclose(drift[0], fd, rtol=1e-6, atol=1e-6)
    assert kin[0] == pytest.approx(-0.5 * lap_sum, rel=1e-5)


def test_exchange_antisymmetry_and_two_by_two():
    mil, coef = shell_orbitals(4)
    rng = np.random.default_rng(8)
    pos = rng.uniform(0, 6, (8, 3))          # one walker: 4 up, 4 down
    ld, s, kin, drift = _logdet(mil, coef, pos, 8, 4)
    swapped = pos.copy()
    swapped[[1, 3]] = swapped[[3, 1]]         # two up electrons
    ld2, s2, kin2, drift2 = _logdet(mil, coef, swapped, 8, 4)
    assert ld2[0] == pytest.approx(ld[0], abs=1e-12) and s2[0] == -s[0]
    assert kin2[0] == pytest.approx(kin[0], rel=1e-12)
    np.testing.assert_allclose(drift2[0][[3, 1]], drift[0][[1, 3]], atol=1e-12)
    # 2 x 2 by hand: D = phi1(r1) phi2(r2) - phi2(r1) phi1(r2)
    v, g, l = outputs(mil, coef, pos[:2])
    D = v[0, 0] * v[1, 1] - v[0, 1] * v[1, 0]
    lapD = l[0, 0] * v[1, 1] - l[0, 1] * v[1, 0] + v[0, 0] * l[1, 1] - v[0, 1] * l[1, 0]
    ld1, s1, k1, _ = oracle.slater_kinetic(v, g, l, 1, 2, 2)
    assert ld1[0] == pytest.approx(math.log(abs(D)), abs=1e-12) and s1[0] == np.sign(D)
    assert k1[0] == pytest.approx(-0.5 * lapD / D, rel=1e-12)


# ---------------------------------------------------------------------------
# complex orbitals (Bloch functions, Sec. II): complex determinants
# ---------------------------------------------------------------------------

def test_complex_planewave_determinant_kinetic_energy_and_phase():
    """Orbitals exp(i (k+G_j).r) are eigenfunctions of -1/2 lap with eigenvalues |k+G_j|^2/2, so
    T_L = 1/2 sum_j |k+G_j|^2 (real) at every configuration; the determinant's modulus and phase
    agree with a direct product formula for one electron per block."""
    n_up, n_dn = 5, 3
    rng = np.random.default_rng(20)
    B = 2 * np.pi * np.linalg.inv(LAT).T
    kvec = B @ np.array([0.137, -0.291, 0.412])
    gs = []
    while len(gs) < 5:
        g = tuple(int(x) for x in rng.integers(-2, 3, 3))
        if g not in gs:
            gs.append(g)
    kg = np.array([kvec + B @ np.array(g) for g in gs])          # [5, 3]
    W = 4
    pos = rng.uniform(0, 6, (W * (n_up + n_dn), 3))
    ph = np.exp(1j * pos @ kg.T)                                    # [P, 5]
    val = ph
    grad = 1j * kg.T[None, :, :] * ph[:, None, :]
    lap = -np.sum(kg ** 2, axis=1)[None, :] * ph
    logdet, sign, kin, drift = oracle.slater_kinetic(val, grad, lap, W, n_up + n_dn, n_up)
    k2 = np.sum(kg ** 2, axis=1)
    np.testing.assert_allclose(kin, 0.5 * (k2[:n_up].sum() + k2[:n_dn].sum()), rtol=1e-10, atol=1e-10)
    assert np.iscomplexobj(sign) and np.allclose(np.abs(sign), 1.0)
    # one electron per block: det = phi_0(r), so ln|det| = 0 and sign = exp(i (k+G_0).r)
    ld1, sg1, _, d1 = oracle.slater_kinetic(val, grad, lap, W * 4, 2, 1)
    np.testing.assert_allclose(ld1, 0.0, atol=1e-12)
    np.testing.assert_allclose(sg1, ph[0::2, 0] * ph[1::2, 0], rtol=1e-12)
    np.testing.assert_allclose(d1[:, 0], 1j * np.broadcast_to(kg[0], d1[:, 0].shape), rtol=1e-12)


def test_complex_drift_and_kinetic_by_finite_differences():
    """Random complex orbitals (random complex planewave sums): the drift is grad_i ln det and the
    kinetic term -1/2 lap_i det / det summed over i, both by central differences of det."""
    rng = np.random.default_rng(21)
    B = 2 * np.pi * np.linalg.inv(LAT).T
    mil = rng.integers(-2, 3, (9, 3))
    coef = rng.standard_normal((4, 9)) + 1j * rng.standard_normal((4, 9))
    kvec = B @ np.array([0.25, 0.1, -0.3])
    kg = np.array([kvec + B @ m for m in mil])

    def orbitals(r):
        e = np.exp(1j * r @ kg.T)                                   # [P, 9]
        v = e @ coef.T
        g = np.einsum("pg,ga,og->pao", 1j * e, kg, coef)
        l = (e * -np.sum(kg ** 2, axis=1)) @ coef.T
        return v, g, l

    n = 4
    r0 = rng.uniform(0, 6, (n, 3))
    v, g, l = orbitals(r0)
    _, _, kin, drift = oracle.slater_kinetic(v, g, l, 1, n, n)
    det = lambda r: np.linalg.det(orbitals(r)[0][:, :n])
    d0 = det(r0)
    h = 1e-4
    fd_drift = np.zeros((n, 3), dtype=complex)
    lap_sum = 0.0
    for i in range(n):
        for a in range(3):
            rp, rm = r0.copy(), r0.copy()
            rp[i, a] += h
            rm[i, a] -= h
            dp, dm = det(rp), det(rm)
            fd_drift[i, a] = (dp - dm) / (2 * h) / d0
            lap_sum += (dp - 2 * d0 + dm) / h ** 2 / d0
    np.testing.assert_allclose(drift[0], fd_drift, rtol=1e-6, atol=1e-6)
    assert abs(kin[0] - (-0.5 * lap_sum)) < 1e-4 * max(1.0, abs(kin[0]))
