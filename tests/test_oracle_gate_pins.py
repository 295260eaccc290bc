"""Pins of the parity gate itself and the 16^3 brute-force pin of the oracle's B-spline path.

Every GPU parity test ends in oracle.relative_error (the tolerance "relative to the maximum
orbital magnitude": max |test - ref| / max |ref| per output), so the gate is checked here on
hand-computed pairs, on a planted difference of known size, and on cases that a plausible
mistake in it (dividing by the wrong maximum, a signed maximum, a swapped argument order, a
mean in place of a maximum) would let through.  The paper's own accuracy metric (Sec. III A,
relative mean absolute error) is pinned the same way.

The brute-force pin follows the C1 workload (a = 10.26 bohr, 16^3 grid, 8 real orbitals,
E_cut 15 Ha, decay 4): interpolating coefficients from a dense 4096 x 4096 solve of the
periodic interpolation system (Appendix, "Interpolating B-spline coefficients") on grid values
from direct planewave sums, then value, gradient and Laplacian of Eq. (b-splineapproximation)
as sums over every grid point and its periodic images, with no stencil bookkeeping.

The rounding of a table to its storage type (FP32, BF16), which every reduced-precision parity
test applies to the oracle's tables, is pinned on hand-computed values and ties.
"""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs


# ---------------------------------------------------------------------------
# relative_error: max |test - ref| / max |ref|
# ---------------------------------------------------------------------------

def test_relative_error_hand_computed_pairs():
    # |diff| = (0, 0, 1), max |ref| = 4
    assert oracle.relative_error(np.array([1.0, 2.0, 3.0]), np.array([1.0, 2.0, 4.0])) == 0.25
    # the largest |diff| is not where |ref| is largest: (3, 0.5) / 8
    assert oracle.relative_error(np.array([3.0, 8.5]), np.array([0.0, 8.0])) == 3.0 / 8.0
    # 2-D arrays: the maxima run over every element
    t = np.array([[1.0, -2.0], [0.5, 7.0]])
    r = np.array([[1.0, -2.5], [0.5, 6.0]])
    assert oracle.relative_error(t, r) == 1.0 / 6.0
    # identical arrays
    assert oracle.relative_error(r, r.copy()) == 0.0
    # references far below and far above one: the gate is scale-free (powers of two, exact)
    assert oracle.relative_error(np.array([0.25, -0.0625]), np.array([0.25, -0.125])) == 0.25
    for c in (2.0 ** -40, 2.0 ** 40):
        assert oracle.relative_error(c * t, c * r) == 1.0 / 6.0


def test_relative_error_zero_and_empty_reference():
    # all-zero reference: the absolute error is returned
    assert oracle.relative_error(np.array([0.0, -3.0, 2.0]), np.zeros(3)) == 3.0
    assert oracle.relative_error(np.zeros(4), np.zeros(4)) == 0.0
    # empty arrays (no positions)
    assert oracle.relative_error(np.zeros((0, 5)), np.zeros((0, 5))) == 0.0


def test_relative_error_reports_a_planted_difference_exactly():
    """A difference of 2^-23 planted in one element of a seeded array whose largest magnitude
    is exactly 2 must be reported as 2^-24 (powers of two: no rounding anywhere)."""
    rng = np.random.default_rng(71)
    ref = rng.uniform(-1.0, 1.0, size=(257, 3, 13))
    ref[17, 1, 5] = -2.0                       # max |ref| = 2 exactly
    ref[100, 2, 7] = 0.5
    test = ref.copy()
    test[100, 2, 7] += 2.0 ** -23              # exact in binary64
    err = oracle.relative_error(test, ref)
    assert abs(err - 2.0 ** -24) <= 1e-15 * 2.0 ** -24
    # float32 test data is widened before the subtraction: 0.5 + 2^-23 is exact in float32
    err32 = oracle.relative_error(test.astype(np.float32), ref)
    assert abs(err32 - oracle.relative_error(test.astype(np.float32).astype(np.float64), ref)) == 0.0
    assert err32 > 0.0


def test_relative_error_divides_by_the_reference_maximum():
    """Cases that a wrong denominator would pass at a tolerance of 0.5."""
    tol = 0.5
    # an error of 9 on a reference of magnitude 1: dividing by max |test| (= 10) gives 0.9,
    # by max |test| + max |ref| 0.82, by the sum of |ref| ... -- the gate must report 9
    test = np.array([10.0, 1.0, 0.0])
    ref = np.array([1.0, 1.0, 0.0])
    assert oracle.relative_error(test, ref) == 9.0
    # argument order matters: (ref, test) divides by 10
    assert oracle.relative_error(ref, test) == 0.9
    # a signed maximum (np.max(ref) = 1 here) would report 1.0 instead of 0.25
    assert oracle.relative_error(np.array([-4.0, 2.0]), np.array([-4.0, 1.0])) == 0.25
    # a mean of |ref| (= 0.5005) in the denominator would give 0.999: the gate says 0.5
    ref = np.concatenate([[1.0], np.full(999, 0.5)])
    test = ref.copy()
    test[0] += 0.5
    assert oracle.relative_error(test, ref) == 0.5
    # the maximum is taken over this output alone: a Laplacian error of 1 against a Laplacian of
    # magnitude 1 fails even when the values are 1e3 times larger
    lap_ref, lap_test = np.array([1.0, -1.0]), np.array([2.0, -1.0])
    assert oracle.relative_error(lap_test, lap_ref) == 1.0 > tol
    assert oracle.relative_error(np.concatenate([lap_test, [1e3]]), np.concatenate([lap_ref, [1e3]])) < tol


def test_relative_error_of_complex_outputs():
    # |(1 + 1j) - (1 + 0j)| = 1, max |ref| = |3 + 4j| = 5
    t = np.array([1 + 1j, 3 + 4j])
    r = np.array([1 + 0j, 3 + 4j])
    assert oracle.relative_error(t, r) == pytest.approx(0.2, abs=1e-16)
    # a purely imaginary error is not lost
    assert oracle.relative_error(np.array([2 + 0.5j]), np.array([2 + 0j])) == pytest.approx(0.25, abs=1e-16)


def test_relative_mean_absolute_error_hand_computed_pairs():
    """Sec. III A: mean |error| / mean |planewave value|."""
    # mean |err| = 2/3, mean |ref| = 8/3
    assert oracle.relative_mean_absolute_error(np.array([1.0, 2.0, 3.0]), np.array([1.0, 2.0, 5.0])) == \
        pytest.approx(0.25, abs=1e-16)
    # signs of the reference do not cancel (a mean of ref would be 0 here)
    assert oracle.relative_mean_absolute_error(np.array([-1.0, 2.0]), np.array([-1.0, 1.0])) == 0.5
    # a mean, not a maximum: one large error among many exact values
    ref = np.ones(100)
    test = ref.copy()
    test[3] = 11.0
    assert oracle.relative_mean_absolute_error(test, ref) == pytest.approx(0.1, abs=1e-16)


# ---------------------------------------------------------------------------
# brute force on 16^3 (the C1 workload)
# ---------------------------------------------------------------------------

def _b(xi):
    """Grid-centred cubic B-spline, Eq. (bsplinegridcenteredbasis), and its first two
    derivatives, written out per branch."""
    a = abs(xi)
    s = 1.0 if xi >= 0 else -1.0
    if a < 1:
        return 0.75 * a ** 3 - 1.5 * a * a + 1.0, s * (2.25 * a * a - 3.0 * a), 4.5 * a - 3.0
    if a < 2:
        return 0.25 * (2 - a) ** 3, -s * 0.75 * (2 - a) ** 2, 1.5 * (2 - a)
    return 0.0, 0.0, 0.0


def _axis_weights(u, n):
    """Weights of every grid point l = 0 .. n-1 on one axis at grid coordinate u, summed over
    the periodic images l + k n (k = -2 .. 2): value, first and second derivative in u."""
    w = np.zeros((3, n))
    for l in range(n):
        for k in range(-2, 3):
            w[:, l] += _b(u - l - k * n)
    return w


def test_c1_brute_force_16_cubed_dense_solve_and_full_grid_sum():
    w = inputs.make_workload("c1", n_pos=24)
    lat, mil, coef, dims = w.lattice, w.miller, w.coef, w.cell.grid
    n_orb = coef.shape[0]
    N = np.array(dims)
    # grid values by direct planewave sums (pinned by the single-planewave closed forms)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, 3)
    gpts = (idx / N) @ lat.T
    phi, _, _, _ = oracle.pw_eval(lat, mil, coef, gpts)            # [4096, 8]
    # the periodic interpolation matrix of one axis, M[i, l] = b(i - l) over all images,
    # and the 4096 x 4096 system as its Kronecker cube
    M = np.zeros((dims[0], dims[0]))
    for i in range(dims[0]):
        M[i] = _axis_weights(float(i), dims[0])[0]
    assert np.allclose(np.diag(M), 1.0) and np.allclose(M.sum(1), 1.5)
    K = np.kron(np.kron(M, M), M)
    beta_dense = np.linalg.solve(K, phi).reshape(dims + (n_orb,))
    beta, _ = oracle.interpolating_tables(lat, mil, coef, dims)
    np.testing.assert_allclose(beta, beta_dense, atol=1e-12 * np.abs(beta_dense).max())

    # value, reduced derivatives and Laplacian at positions inside and outside the cell
    pos = np.concatenate([w.pos[:12], inputs.positions(lat, 12, 77, -2.0, 3.0)])
    ainv = np.linalg.inv(lat)
    metric = ainv @ ainv.T                                          # (a^-1 a^-T)
    bv = np.zeros((len(pos), n_orb))
    bg = np.zeros((len(pos), 3, n_orb))
    bl = np.zeros((len(pos), n_orb))
    for p, r in enumerate(pos):
        s = ainv @ r
        u = (s - np.floor(s)) * N
        wx, wy, wz = (_axis_weights(u[a], dims[a]) for a in range(3))

        def contract(dx, dy, dz):
            return np.einsum("i,j,k,ijko->o", wx[dx], wy[dy], wz[dz], beta_dense)

        bv[p] = contract(0, 0, 0)
        gs = np.array([contract(1, 0, 0), contract(0, 1, 0), contract(0, 0, 1)]) * N[:, None]   # d/ds
        bg[p] = ainv.T @ gs
        H = np.zeros((3, 3, n_orb))
        for i in range(3):
            for j in range(3):
                d = [0, 0, 0]
                d[i] += 1
                d[j] += 1
                H[i, j] = contract(*d) * N[i] * N[j]
        bl[p] = np.einsum("ij,ijo->o", metric, H)
    val, grad, lap = oracle.bspline_eval(beta, lat, pos)
    assert oracle.relative_error(val, bv) < 1e-12
    assert oracle.relative_error(grad, bg) < 1e-12
    assert oracle.relative_error(lap, bl) < 1e-12
    # the interpolating spline passes through the planewave grid values
    gv, _, _ = oracle.bspline_eval(beta, lat, gpts[::97])
    assert oracle.relative_error(gv, phi[::97]) < 1e-12


# ---------------------------------------------------------------------------
# storage rounding: one round-to-nearest-even from FP64 to FP32 or BF16
# ---------------------------------------------------------------------------

def test_round_to_storage_hand_computed_and_ties_to_even():
    r = oracle.round_to_storage
    # BF16 keeps 8 significant bits: the spacing above 1 is 2^-7
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -30, -(1.0 + 2.0 ** -8),
                  0.0, 3.0, 255.5, 2.0 ** -100, -6.5])
    want = np.array([1.0, 1.0, 1.0 + 2 * 2.0 ** -7, 1.0 + 2.0 ** -7, -1.0, 0.0, 3.0, 256.0, 2.0 ** -100, -6.5])
    np.testing.assert_array_equal(r(x, "bf16"), want)
    # FP32: 24 significant bits, ties to even, against numpy's own IEEE conversion
    rng = np.random.default_rng(72)
    y = rng.standard_normal(100_000) * np.exp(rng.uniform(-20, 20, 100_000))
    y[:4] = [1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -60, 0.1]
    np.testing.assert_array_equal(r(y, "f32"), y.astype(np.float32).astype(np.float64))
    assert r(y, "f64") is y and r(None, "bf16") is None


def test_round_to_storage_bf16_is_a_single_rounding():
    """BF16 of a float64 value is rounded once: values just above a BF16 midpoint round up even
    when their nearest float32 is the midpoint itself (rounding through float32 first would round
    those to even, i.e. down, one BF16 step off)."""
    r = oracle.round_to_storage
    mid = 1.0 + 2.0 ** -8                      # halfway between 1 and 1 + 2^-7
    x = np.array([mid + 2.0 ** -30, mid - 2.0 ** -30])
    assert float(x[0].astype(np.float32)) == mid   # float32 cannot tell them from the midpoint
    np.testing.assert_array_equal(r(x, "bf16"), [1.0 + 2.0 ** -7, 1.0])
    # the result is representable in BF16: its FP32 bits have 16 zero low bits
    rng = np.random.default_rng(73)
    z = r(rng.standard_normal(10_000), "bf16").astype(np.float32)
    assert np.all(z.view(np.uint32) & 0xFFFF == 0)
    # and it is the nearest such value: within half a BF16 step of the input
    w = rng.standard_normal(10_000)
    q = r(w, "bf16")
    assert np.all(np.abs(q - w) <= 0.5 * np.ldexp(1.0, np.frexp(q)[1] - 8) + 1e-300)
