"""The product's host post-processing of the two-step current
(``paper_2112_00920_gb300/twostep.py``: eps(omega) of Eqs. 12-14 and the
standard error of the shift mean of Sec. III.B) against the oracle's
independent implementations, on seeded synthetic current histories.  No GPU
is used; the two sides share no code."""
import numpy as np
import pytest

from oracle import analysis


def _histories(n_h, n_t, seed):
    rng = np.random.default_rng([seed, 31])
    t = np.arange(n_t) * 0.08
    base = 1e-4 * np.sin(0.3 * t) * np.exp(-0.01 * t)
    return base[None, :] + 1e-6 * rng.standard_normal((n_h, n_t))


@pytest.mark.parametrize("t_w", [None, 30.0])
def test_dielectric_matches_oracle(t_w):
    from paper_2112_00920_gb300 import twostep
    dj = _histories(1, 501, 1)[0]
    om = np.linspace(0.01, 0.7, 97)
    got = twostep.dielectric(dj, 0.08, 0.005, om, t_w=t_w)
    ref = analysis.dielectric(dj, 0.08, 0.005, om, t_w=t_w)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n_h", [1, 2, 7])
def test_standard_error_of_eps_matches_oracle(n_h):
    from paper_2112_00920_gb300 import twostep
    dj = _histories(n_h, 401, 2 + n_h)
    om = np.linspace(0.02, 0.6, 41)
    eps = np.stack([twostep.dielectric(d, 0.08, 0.005, om) for d in dj])
    mean, s_re, s_im = twostep.standard_error(eps)
    r_mean, r_re, r_im = analysis.dielectric_statistics(dj, 0.08, 0.005, om)
    scale = np.max(np.abs(r_mean))
    np.testing.assert_allclose(mean, r_mean, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(s_re, r_re, rtol=1e-9, atol=1e-15 * scale)
    np.testing.assert_allclose(s_im, r_im, rtol=1e-9, atol=1e-15 * scale)
    if n_h == 1:
        assert not np.any(s_re) and not np.any(s_im)
