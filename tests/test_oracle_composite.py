"""Pins of the composite mass class (Sect. 3.3, kappa_int,comp; Eqs. Chameleon, kappa_enfw;
App. B) in the oracle: the softened isothermal and CSE potentials and Jacobians against
differences of their deflections, the complex NFW profile on the real axis, the black-hole
Gaussian lens against differences and Gauss's theorem, the round composite galaxy against
Gauss's theorem on its exact convergence (baryons + exact NFW + black hole) by quadrature, the
class's potential <-> deflection <-> Jacobian with the sheet, the 1-D MGEs (halo alone and the
whole mass model) against the profiles, and the ideal-sheet transform of the composite image."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import chameleon, enfw, imaging, lensmodel, mge, model
from paper_2504_01302_b300 import synth

from . import systems

I = synth.IDX


def _comp_system(**kw):
    return synth.composite_light(dict(systems.small_base(7), **kw))


@pytest.mark.parametrize("q,s", [(0.65, 0.3), (1.0, 0.2), (0.4, 2.0)])
def test_nie_and_cse_potential_and_jacobian(q, s):
    h = 1e-6
    for x, y in ((0.4, -0.9), (1.7, 0.3)):
        for al, ps, jc in ((lambda a, b: chameleon._nie_alpha(a, b, 1.3, s, q),
                            lambda a, b: chameleon._nie_psi(a, b, 1.3, s, q),
                            lambda a, b: chameleon._nie_jac(a, b, 1.3, s, q)),
                           (lambda a, b: enfw.cse_alpha(a, b, s, q),
                            lambda a, b: enfw.cse_psi(a, b, s, q),
                            lambda a, b: enfw.cse_jac(a, b, s, q))):
            A = lambda a, b: np.array(al(np.array([a]), np.array([b])))[:, 0]
            P = lambda a, b: ps(np.array([a]), np.array([b]))[0]
            ax, ay = A(x, y)
            sc = max(abs(ax), abs(ay))
            assert abs((P(x + h, y) - P(x - h, y)) / (2 * h) - ax) < 1e-8 * max(1.0, sc)
            assert abs((P(x, y + h) - P(x, y - h)) / (2 * h) - ay) < 1e-8 * max(1.0, sc)
            J = jc(np.array([x]), np.array([y]))
            dx = (A(x + h, y) - A(x - h, y)) / (2 * h)
            dy = (A(x, y + h) - A(x, y - h)) / (2 * h)
            ref = np.array([dx[0], dy[0], dx[1], dy[1]])
            got = np.array([J[0][0], J[1][0], J[2][0], J[3][0]])
            assert np.max(np.abs(got - ref)) < 1e-7 * max(1.0, np.max(np.abs(ref)))


def test_complex_nfw_profile():
    u = np.array([1e-3, 0.3, 0.9, 0.95, 0.99, 1.0, 1.01, 1.05, 1.1, 3.0, 40.0])
    k = enfw.nfw_k_complex(u)
    assert np.max(np.abs(k.imag)) == 0.0
    assert np.allclose(k.real, enfw.nfw_k(u), rtol=1e-12, atol=0)
    # continuous across the switch to the Taylor branch (|w| = 0.1) at complex arguments
    for ph in (0.3, 1.2, 2.5):
        w = 0.1 * np.exp(1j * ph) * np.array([1 - 1e-9, 1 + 1e-9])
        uu = np.sqrt(1 - w * w)
        kk = enfw.nfw_k_complex(uu)
        assert abs(kk[0] - kk[1]) < 1e-9


def test_gaussian_lens_is_gauss():
    M, sg = 0.03, 0.01
    for R in (0.0, 2e-4, 0.01, 0.05, 1.0):
        (ax, ay), _, J = lensmodel.gauss_lens(np.array([0.6 * R]), np.array([0.8 * R]), M, sg)
        mass = M * -math.expm1(-R * R / (2 * sg * sg))
        assert abs(math.hypot(ax[0], ay[0]) - (mass / (math.pi * R) if R > 0 else 0.0)) < 1e-12
        S0 = M / (2 * math.pi * sg * sg)
        assert abs(J[0][0] + J[3][0] - 2 * S0 * math.exp(-R * R / (2 * sg * sg))) < 1e-9 * S0


def test_round_composite_galaxy_is_gauss():
    """Round Chameleons, round halo, no shear or perturbers: the deflection is R times the mean
    convergence inside R, by quadrature of Upsilon L_scale I + kappa_s k(R/r_s) + the black hole."""
    s = dict(_comp_system(), ll_q=1.0, ll2=np.array([[0.3, 0.3, 3.0, 1.0]]), sis=np.zeros((0, 3)))
    th = synth.theta_truth_composite()
    th[I["q"]] = 1.0
    th[I["gamma_ext"]] = 0.0
    M = lensmodel.bh_mass(th, s)
    assert M > 0
    ups = th[I["upsilon"]] * s["L_scale"]

    def kap(r):
        k = th[0] * enfw.nfw_k(np.array([r / th[1]]))[0]
        for I0, wc, wt, q in lensmodel.chameleons(th, s):
            k += ups * chameleon.kappa(np.array([r]), np.array([0.0]), I0, wc, wt, q)[0]
        return k + M / (2 * math.pi * s["bh_sigma"] ** 2) * math.exp(-r * r / (2 * s["bh_sigma"] ** 2))
    # (the CSE fit of the halo holds k(u) to 1e-6 on [1e-4, 1e3]; inside 0.1" the mean
    # convergence also integrates u < 1e-4, where the fit's error reaches ~1e-4)
    for R, tol in ((0.02, 2e-4), (0.4, 1e-5), (1.65, 1e-5), (5.0, 1e-5)):
        brk = [p for p in (0.01, 0.05, 0.3) if p < R]
        m = 2 * math.pi * quad(lambda r: r * kap(r), 1e-6, R, epsabs=0, epsrel=1e-12, limit=400,
                               points=brk or None)[0]
        (ax, ay), _, _ = lensmodel.composite_galaxy(np.array([0.6 * R]), np.array([0.8 * R]), th, s)
        assert abs(math.hypot(ax[0], ay[0]) / (m / (math.pi * R)) - 1) < tol, R


@pytest.mark.parametrize("lam", [1.0, 0.85])
def test_composite_class_potential_deflection_jacobian(lam):
    s = _comp_system(sheet=1 if lam != 1.0 else 0)
    th = synth.theta_truth_composite()
    th[I["lam_int"]] = lam
    h = 1e-5
    for x, y in ((0.9, -1.2), (-1.4, 0.6), (0.05, 0.02)):
        P = lambda a, b: lensmodel.psi(np.array([a]), np.array([b]), th, s)[0]
        A = lambda a, b: np.array(lensmodel.alpha(np.array([a]), np.array([b]), th, s))[:, 0]
        ax, ay = A(x, y)
        assert abs((P(x + h, y) - P(x - h, y)) / (2 * h) - ax) < 1e-6
        assert abs((P(x, y + h) - P(x, y - h)) / (2 * h) - ay) < 1e-6
        J = lensmodel.jac(np.array([x]), np.array([y]), th, s)
        dx = (A(x + h, y) - A(x - h, y)) / (2 * h)
        dy = (A(x, y + h) - A(x, y - h)) / (2 * h)
        assert np.allclose([J[0][0], J[1][0], J[2][0], J[3][0]], [dx[0], dy[0], dx[1], dy[1]],
                           atol=1e-6, rtol=1e-6)


def test_halo_and_mass_mge_reconstruct_the_profiles():
    # an MGE of realistic size (the test systems' 8 and 5 + 4 Gaussians are too coarse for it)
    # on a range wide enough for the halo: with r_s = 23" much of its convergence inside 10"
    # comes from Gaussians wider than the 50" the workloads use (the paper's MGE extent), and
    # dropping them leaves a near-constant deficit of a few per cent there
    s = synth.composite_light(dict(systems.small_base(7, n_mass=40, n_light=(24, 24)),
                                   mass_rmax=5000.0))
    th = synth.theta_truth_composite()
    A, sg, q = lensmodel.enfw_mass_mge(th, s)
    R = np.geomspace(0.05, 10.0, 40)
    ref = th[0] * enfw.nfw_k(R / th[1])
    assert np.max(np.abs(mge.mge_eval(R, sg, A) / ref - 1)) < 5e-3
    # the whole mass model along the major axis (halo + Upsilon x the Chameleon light)
    tr = model.light_mge(th, s)
    ms = model.mass_mge(th, dict(s, has_bh=False), 1.0, tr)
    ups = th[I["upsilon"]] * s["L_scale"]
    # along the major axis each Gaussian's own axis ratio does not enter
    got = mge.mge_eval(R, ms["sig"], ms["kap0"])
    bar = sum(ups * chameleon.kappa(R, 0 * R, I0, wc, wt, qq) for I0, wc, wt, qq in lensmodel.chameleons(th, s))
    assert np.max(np.abs(got / (ref + bar) - 1)) < 5e-3


def test_ideal_sheet_transform_of_the_composite_image():
    s = _comp_system(sheet=2)
    s.update(data=np.zeros((s["ny"], s["nx"])), img_xy=np.zeros((4, 2)))
    th = synth.theta_truth_composite()
    th[I["lam_int"]] = 1.0
    m0 = imaging.model_image(th, s)
    lam = 0.8
    t2 = th.copy()
    t2[I["lam_int"]] = lam
    t2[I["x_src"]] = lam * th[I["x_src"]] + (1 - lam) * th[I["x_c"]]
    t2[I["y_src"]] = lam * th[I["y_src"]] + (1 - lam) * th[I["y_c"]]
    t2[I["R_e_src"]] = lam * th[I["R_e_src"]]
    assert np.max(np.abs(imaging.model_image(t2, s) - m0)) <= 1e-12 * np.max(np.abs(m0))
