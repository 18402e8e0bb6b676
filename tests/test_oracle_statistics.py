"""Pins of the oracle's shift statistics (error bars of Fig. 6, Sec. III.B):
the standard error of the two-step mean over N_H sub-simulations, for the
current and for eps(omega).  Closed forms on synthetic per-shift data; no
propagation."""
import numpy as np

from oracle import analysis, dynamics


def _results(dj_list):
    # per-shift results with J(0-) folded in: dJ = J - J(0-)
    out = []
    for m, d in enumerate(dj_list):
        j0 = np.array([0.1 * m, -0.2, 0.3 + m])
        out.append({"J": d + j0[None, :], "J0_minus": j0})
    return out


def test_two_shifts_half_difference():
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=(7, 3)), rng.normal(size=(7, 3))
    mean, se = dynamics.two_step_standard_error(_results([a, b]))
    np.testing.assert_allclose(mean, 0.5 * (a + b), rtol=0, atol=1e-15)
    np.testing.assert_allclose(se, 0.5 * np.abs(a - b), rtol=1e-14, atol=1e-16)


def test_arithmetic_sequence_closed_form():
    # dJ_m = m c, m = 1..N: sample variance N(N+1)/12 c^2, standard error |c| sqrt((N+1)/12)
    c = np.array([[1.5, -0.25, 2.0], [0.5, 3.0, -1.0]])
    for n in (2, 3, 10, 64):
        mean, se = dynamics.two_step_standard_error(_results([m * c for m in range(1, n + 1)]))
        np.testing.assert_allclose(mean, 0.5 * (n + 1) * c, rtol=1e-14)
        np.testing.assert_allclose(se, np.abs(c) * np.sqrt((n + 1) / 12.0), rtol=1e-13)


def test_identical_and_single_shift():
    d = np.arange(12.0).reshape(4, 3)
    mean, se = dynamics.two_step_standard_error(_results([d, d, d]))
    np.testing.assert_allclose(mean, d, rtol=0, atol=1e-13)
    assert np.all(se <= 1e-14)
    mean, se = dynamics.two_step_standard_error(_results([d]))
    np.testing.assert_array_equal(se, 0.0)
    np.testing.assert_allclose(mean, d, atol=1e-15)


def test_mean_is_the_two_step_average():
    rng = np.random.default_rng(5)
    res = _results([rng.normal(size=(9, 3)) for _ in range(5)])
    mean, _ = dynamics.two_step_standard_error(res)
    np.testing.assert_allclose(mean, dynamics.two_step_average(res), rtol=1e-14, atol=1e-16)


def test_dielectric_statistics_affine():
    # eps is affine in dJ: per-shift dJ_m = base + m delta gives the mean eps of the
    # mean dJ, and error bars |Re / Im of the linear part of delta| sqrt((N+1)/12)
    dt, k0, n_t = 0.08, 0.005, 400
    t = np.arange(n_t + 1) * dt
    base = 1e-3 * np.sin(0.3 * t) * np.exp(-0.01 * t)
    delta = 2e-5 * np.cos(0.7 * t)
    om = np.linspace(0.01, 0.7, 50)
    n = 6
    djs = np.stack([base + m * delta for m in range(1, n + 1)])
    mean, sre, sim = analysis.dielectric_statistics(djs, dt, k0, om)
    ref = analysis.dielectric(djs.mean(axis=0), dt, k0, om)
    np.testing.assert_allclose(mean, ref, rtol=1e-12, atol=1e-12)
    lin = analysis.dielectric(delta, dt, k0, om) - 1.0
    scale = np.sqrt((n + 1) / 12.0)
    np.testing.assert_allclose(sre, np.abs(lin.real) * scale, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(sim, np.abs(lin.imag) * scale, rtol=1e-9, atol=1e-12)
