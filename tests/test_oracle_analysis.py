"""Pins of the oracle's HHG spectrum (Eqs. 16-17) against closed forms.

I(w) = w^2 |int_0^T dt e^{iwt} W(t) J(t)|^2 with W(t) = sin^4(pi t/T).
For a test current that is a sum of complex exponentials the integral is
exact in closed form: sin^4(x) = 3/8 - cos(2x)/2 + cos(4x)/8 turns the
integrand into a sum of terms c e^{i alpha t}, each integrating to
c (e^{i alpha T} - 1)/(i alpha).  The window vanishes at both ends together
with its first three derivatives, so the trapezoid sum of the oracle agrees
with the integral to O(dt^6) (Euler-Maclaurin).  A dropped w^2, a wrong
power or argument of the window, a missing dt or a flipped sign of the
exponent (seen with a one-sided complex test signal) fails these checks.
"""
import numpy as np

from oracle import analysis


def _exp_integral(alpha, t_end):
    alpha = np.asarray(alpha, dtype=np.float64)
    out = np.empty(alpha.shape, dtype=np.complex128)
    small = np.abs(alpha) < 1e-14
    out[small] = t_end
    a = alpha[~small]
    out[~small] = (np.exp(1j * a * t_end) - 1.0) / (1j * a)
    return out


def _windowed_transform(omegas, terms, t_end):
    """int_0^T e^{iwt} sin^4(pi t/T) sum_j c_j e^{i b_j t} dt in closed form."""
    om = np.pi / t_end
    window = [(3.0 / 8.0, 0.0), (-0.25, 2.0 * om), (-0.25, -2.0 * om), (1.0 / 16.0, 4.0 * om),
              (1.0 / 16.0, -4.0 * om)]
    total = np.zeros(omegas.shape, dtype=np.complex128)
    for cw, fw in window:
        for cj, bj in terms:
            total += cw * cj * _exp_integral(omegas + fw + bj, t_end)
    return total


def test_hhg_spectrum_single_frequency_closed_form():
    """J(t) = sin(w1 t + phi): closed-form intensity, peak at w1."""
    t_end, dt, w1, phi = 200.0, 0.05, 0.5, 0.3
    n = int(round(t_end / dt))
    t = np.arange(n + 1) * dt
    j = np.sin(w1 * t + phi)
    omegas = np.linspace(0.05, 1.5, 300)
    got = analysis.hhg_spectrum(j, dt, t_end, omegas)
    terms = [(np.exp(1j * phi) / 2j, w1), (-np.exp(-1j * phi) / 2j, -w1)]
    ref = omegas ** 2 * np.abs(_windowed_transform(omegas, terms, t_end)) ** 2
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * ref.max())
    assert abs(omegas[np.argmax(got)] - w1) < 2 * (omegas[1] - omegas[0])


def test_hhg_spectrum_harmonics_and_exponent_sign():
    """A current with a fundamental and a weak 3rd harmonic: both peaks and
    their ratio follow the closed form.  A one-sided complex signal
    e^{-i w1 t} has its weight at w = +w1 with the e^{+iwt} convention of
    Eq. 16, and none at -w1."""
    t_end, dt, w1 = 300.0, 0.04, 0.4
    n = int(round(t_end / dt))
    t = np.arange(n + 1) * dt
    j = np.cos(w1 * t) + 1e-3 * np.cos(3 * w1 * t + 0.7)
    omegas = np.linspace(0.1, 1.6, 500)
    got = analysis.hhg_spectrum(j, dt, t_end, omegas)
    terms = [(0.5, w1), (0.5, -w1), (0.5e-3 * np.exp(0.7j), 3 * w1), (0.5e-3 * np.exp(-0.7j), -3 * w1)]
    ref = omegas ** 2 * np.abs(_windowed_transform(omegas, terms, t_end)) ** 2
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * ref.max())
    i1, i3 = np.argmin(np.abs(omegas - w1)), np.argmin(np.abs(omegas - 3 * w1))
    assert got[i3] / got[i1] > 0.5 * (3e-3) ** 2   # (3 w1)^2 / w1^2 times the amplitude ratio squared
    # sign of the exponent
    z = np.exp(-1j * w1 * t)
    pm = np.array([w1, -w1])
    gz = analysis.hhg_spectrum(z, dt, t_end, pm)
    refz = pm ** 2 * np.abs(_windowed_transform(pm, [(1.0, -w1)], t_end)) ** 2
    np.testing.assert_allclose(gz, refz, rtol=0, atol=1e-9 * refz.max())
    assert gz[0] > 1e6 * gz[1]


def test_hhg_spectrum_window_zero_outside_pulse():
    """Samples at or after T_L do not contribute (W = 0 outside (0, T_L))."""
    t_end, dt = 100.0, 0.05
    n = int(round(1.5 * t_end / dt))
    t = np.arange(n + 1) * dt
    j = np.sin(0.7 * t)
    j2 = j.copy()
    j2[t >= t_end] = 123.0
    om = np.linspace(0.2, 1.2, 50)
    np.testing.assert_array_equal(analysis.hhg_spectrum(j, dt, t_end, om), analysis.hhg_spectrum(j2, dt, t_end, om))
