"""Post-processing (paper_2504_01302_b300/post.py): BIC weights and H0 from the distance
posterior, against closed forms, brute-force convolution and the oracle's distances
(pinned to Table 2)."""
import math

import numpy as np
from scipy.integrate import quad
from scipy.stats import norm

from oracle import cosmo
from paper_2504_01302_b300 import post


def test_bic_definition():
    # k ln n - 2 ln L with ln L = -chi^2/2
    assert abs(post.bic(48.0, 20, 50) - (20 * math.log(50) + 48.0)) < 1e-12


def test_bic_weights_plain():
    b = np.array([110.0, 100.0, 104.0])
    w = post.bic_weights(b)
    ref = np.exp(-0.5 * (b - 100.0))
    assert np.allclose(w, ref / ref.sum(), rtol=1e-14)
    assert np.allclose(post.bic_weights([7.0, 7.0, 7.0]), 1.0 / 3.0)


def test_bic_weights_convolved_match_brute_force():
    # f* = (f conv N(0, s^2)) with f(D) = 1 for D <= 0, exp(-D/2) above, by quadrature
    s = 3.0
    b = np.array([100.0, 101.5, 106.0, 112.0])

    def fstar(d):
        f = lambda x: (1.0 if d - x <= 0 else math.exp(-0.5 * (d - x))) * norm.pdf(x, 0.0, s)
        return quad(f, -60.0, 60.0, points=[d], epsabs=0, epsrel=1e-12, limit=200)[0]
    ref = np.array([fstar(d) for d in b - b.min()])
    assert np.allclose(post.bic_weights(b, s), ref / ref.sum(), rtol=1e-9)
    # vanishing scatter returns the plain weights
    assert np.allclose(post.bic_weights(b, 1e-6), post.bic_weights(b), rtol=1e-6)


def test_distances_match_oracle():
    for H0, om in ((82.5, 0.27), (60.0, 0.1), (110.0, 0.45)):
        D_d, _, _, D_dt = cosmo.distances(0.295, 0.654, H0, om)
        d, t = post.flat_lcdm_distances(0.295, 0.654, np.array([H0]), np.array([om]))
        assert abs(d[0] / D_d - 1) < 1e-12 and abs(t[0] / D_dt - 1) < 1e-12


def test_h0_recovered_from_synthetic_chain():
    # a chain around the truth distances (H0 82.5, Om 0.27, kappa_ext 0) with 2 % / 4 %
    # scatter gives H0 near 82.5; the D_dt marginal alone gives a wider interval
    D_d, _, _, D_dt = cosmo.distances(0.295, 0.654, 82.5, 0.27)
    rng = np.random.Generator(np.random.PCG64(5))
    ddt = D_dt * (1 + 0.02 * rng.standard_normal(1500))
    dd = D_d * (1 + 0.04 * rng.standard_normal(1500))
    both = post.h0_posterior(ddt, dd, 0.295, 0.654, n=40000, seed=1)
    only = post.h0_posterior(ddt, dd, 0.295, 0.654, use="ddt", n=40000, seed=1)
    assert abs(both["median"] - 82.5) < 1.5
    assert both["lo"] < 82.5 < both["hi"]
    assert (only["hi"] - only["lo"]) > (both["hi"] - both["lo"])
    # a chain of D_dt,int = 0.9 D_dt read with kappa_ext = 0.1 in the draws (Eq. Dt external
    # internal) gives the H0 of the unscaled chain read without it
    k = post.h0_posterior(ddt * 0.9, dd, 0.295, 0.654, kappa_ext_draws=[0.1], use="ddt",
                          n=40000, seed=1)
    assert abs(k["median"] / only["median"] - 1) < 0.02
