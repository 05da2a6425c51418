"""Pins of the spherically aligned Jeans model of the oracle (oracle/jam_sph.py).

The solution is derived from Eqs. J1/J2 (Sect. 3.2); these tests tie it to things other
than itself:
* it satisfies J1 and J2 (central differences of the plain solution, flattened tracer and
  mass, beta of both signs);
* at beta = 0 it is the isotropic solution, which any alignment shares: nu v_z^2 and
  nu v_phi^2 of the cylindrical Jeans equations (jam.PlainJeans, written independently);
* with every Gaussian round the projected rule matches the textbook projection of the
  spherical constant-beta Jeans equation (Binney & Mamon 1982), written out here by
  nested quadrature;
* at beta = 0 the projected rule matches the cylindrical pair form (jam.table) on the
  RXJ1131-scale sky grid, to the rule's discretisation error;
* the discrete grid values match the plain solution;
* Sigma v^2 scales with the mass, is independent of the tracer amplitude (as a ratio to
  Sigma) and is 4-fold symmetric on the sky."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erf

from oracle import jam, jam_sph, model
from paper_2504_01302_b300 import synth

from . import systems


@pytest.fixture(scope="module")
def w0():
    sys_list, th, _ = systems.workload(0)
    s = sys_list[0]
    st, d = model.dynamics_setup(th[0], s)
    assert st == model.ST_OK
    return s, th[0], d


def test_plain_solution_satisfies_jeans_equations(w0):
    s, th, d = w0
    inc = th[synth.IDX["inc"]]
    for beta in (0.25, -0.2):
        m = jam_sph.SphModel(d["tr"], d["ms"], inc, beta, d["v2u"])
        for r, t in ((0.3, 0.7), (1.1, 1.2)):
            h = 1e-4
            P, D = jam_sph.intrinsic_plain(m, r, t)
            Pr = (jam_sph.intrinsic_plain(m, r * (1 + h), t)[0] -
                  jam_sph.intrinsic_plain(m, r * (1 - h), t)[0]) / (2 * r * h)
            Pt = (jam_sph.intrinsic_plain(m, r, t + h)[0] - jam_sph.intrinsic_plain(m, r, t - h)[0]) / (2 * h)
            R, z = r * math.sin(t), r * math.cos(t)
            V = (1 - beta) * P + R * R * D
            nu = float(m.tracer(R * R, z * z)[0])
            dPr, dPt = jam_sph.phi_derivs(m, r, t)
            j1 = Pr + ((1 + beta) * P - V) / r + nu * dPr
            j2 = (1 - beta) * Pt + ((1 - beta) * P - V) / math.tan(t) + nu * dPt
            assert abs(j1) <= 1e-6 * abs(nu * dPr), (beta, r, t, j1 / (nu * dPr))
            assert abs(j2) <= 1e-6 * abs(nu * dPt), (beta, r, t, j2 / (nu * dPt))


def test_isotropic_limit_equals_cylindrical_solution(w0):
    s, th, d = w0
    inc = th[synth.IDX["inc"]]
    m = jam_sph.SphModel(d["tr"], d["ms"], inc, 0.0, d["v2u"])
    pj = jam.PlainJeans(d["tr"], d["ms"], inc, 0.0, d["v2u"])
    for r, t in ((0.3, 0.7), (0.05, 0.3), (1.1, 1.45)):
        P, D = jam_sph.intrinsic_plain(m, r, t)
        R, z = r * math.sin(t), r * math.cos(t)
        vz, dvz = pj.nuvz2(R, z)
        vphi = vz + R * dvz + R * pj.nu(R, z) * pj.dphi(R, z)[0]
        assert abs(P / vz - 1) < 1e-9
        assert abs((P + R * R * D) / vphi - 1) < 1e-9


def _round_mges():
    sig_l = np.geomspace(0.02, 4.0, 8)
    sig_m = np.geomspace(0.01, 8.0, 9)
    tr = dict(I0=3.0 * sig_l ** -1.2, sig=sig_l, qp=np.ones_like(sig_l))
    ms = dict(kap0=0.8 * sig_m ** -0.9, sig=sig_m, qp=np.ones_like(sig_m))
    return tr, ms


def _textbook(Rp, beta, tr, ms, v2u):
    """Sigma v_los^2(R) = 2 int_R^inf (1 - beta R^2/r^2) nu sigma_r^2 r dr / sqrt(r^2 - R^2),
    nu sigma_r^2(r) = int_r^inf (r'/r)^(2 beta) nu(r') G M(r') / r'^2 dr' (spherical Jeans
    equation with constant beta), with r = R cosh(t)."""
    nu0 = tr["I0"] / (math.sqrt(2 * math.pi) * tr["sig"])
    rho0 = ms["kap0"] / (math.sqrt(2 * math.pi) * ms["sig"])
    Mj = (2 * math.pi) ** 1.5 * rho0 * ms["sig"] ** 3
    top = 60.0 * float(np.max(tr["sig"]))

    def nu(r):
        return float(np.sum(nu0 * np.exp(-r * r / (2 * tr["sig"] ** 2))))

    def GM(r):
        x = r / ms["sig"]
        return v2u * float(np.sum(Mj * (erf(x / math.sqrt(2)) - math.sqrt(2 / math.pi) * x * np.exp(-x * x / 2))))

    def nusr2(r):
        f = lambda rp: (rp / r) ** (2 * beta) * nu(rp) * GM(rp) / (rp * rp)
        return quad(f, r, top, epsabs=0, epsrel=1e-11, limit=400)[0]

    def outer(t):
        r = Rp * math.cosh(t)
        return (1 - beta / math.cosh(t) ** 2) * nusr2(r) * r

    tmax = math.acosh(top / Rp)
    return 2 * quad(outer, 0.0, tmax, epsabs=0, epsrel=1e-9, limit=400)[0]


def test_spherical_limit_matches_textbook_projection():
    tr, ms = _round_mges()
    v2u, inc, beta = 1.7e4, 0.9, 0.3
    m = jam_sph.SphModel(tr, ms, inc, beta, v2u)
    rule = jam_sph.SphRule(tr["sig"], ms["sig"], 0.02, 160, 4, 128, 48)
    g = jam_sph.grid_moments(m, rule)
    for Rp, ang in ((0.05, 0.3), (0.3, 1.1), (1.0, 2.5)):
        got = jam_sph.sigma_v2_sph([Rp * math.cos(ang)], [Rp * math.sin(ang)], m, rule, g)[0]
        ref = _textbook(Rp, beta, tr, ms, v2u)
        assert abs(got / ref - 1) < 2e-4, (Rp, got, ref)


def test_beta0_projection_matches_cylindrical_pair_form():
    sys_list, _, _ = systems.workload(1)
    s = sys_list[0]
    t = synth.theta_truth(1).copy()
    t[synth.IDX["beta"]] = 0.0
    st, d = model.dynamics_setup(t, s)
    assert st == model.ST_OK
    rng = np.random.Generator(np.random.PCG64(3))
    sel = rng.choice(d["xp"].size, 200, replace=False)
    X, Y = d["xp"].ravel()[sel], d["yp"].ravel()[sel]
    ref = jam.sigma_v2_fast(X, Y, d["tab"])
    m = jam_sph.SphModel(d["tr"], d["ms"], t[synth.IDX["inc"]], 0.0, d["v2u"])
    rule = model.sph_rule(dict(s, jam_align=1), d["tr"]["sig"], d["ms"]["sig"])
    got = jam_sph.sigma_v2_sph(X, Y, m, rule, jam_sph.grid_moments(m, rule))
    # the default rule's discretisation error (2.9e-4 measured); it falls as n_r^-3.3
    assert np.max(np.abs(got / ref - 1)) < 1e-3


def test_grid_values_match_plain_solution(w0):
    s, th, d = w0
    m = jam_sph.SphModel(d["tr"], d["ms"], th[synth.IDX["inc"]], 0.2, d["v2u"])
    rule = jam_sph.SphRule(d["tr"]["sig"], d["ms"]["sig"], 0.0625, 24, 5, 32, s["n_gl"])
    vr2, dg = jam_sph.grid_moments(m, rule)
    for a, c in ((3, 1), (10, 4), (17, 0), (20, 2)):
        r = math.exp(rule.lr[a])
        t = math.asin(math.sqrt(rule.w[c]))
        P, D = jam_sph.intrinsic_plain(m, r, t, s_max=math.log(rule.r_end / r))
        nu = float(m.tracer(r * r * rule.w[c], r * r * (1 - rule.w[c]))[0])
        assert abs(vr2[a, c] / (P / nu) - 1) < 1e-5, (a, c, vr2[a, c], P / nu)
        assert abs(dg[a, c] - D / nu) < 1e-5 * (abs(D / nu) + abs(vr2[a, c]) / r ** 2), (a, c)


def test_invariants(w0):
    s, th, d = w0
    inc = th[synth.IDX["inc"]]
    tr, ms = d["tr"], d["ms"]
    rule = jam_sph.SphRule(tr["sig"], ms["sig"], 0.0625, 24, 4, 32, s["n_gl"])

    def sv2(tr_, ms_, X, Y):
        m = jam_sph.SphModel(tr_, ms_, inc, 0.15, d["v2u"])
        return jam_sph.sigma_v2_sph(X, Y, m, rule, jam_sph.grid_moments(m, rule))

    X = np.array([0.13, -0.13, 0.13, -0.13, 0.4])
    Y = np.array([0.27, 0.27, -0.27, -0.27, -0.05])
    base = sv2(tr, ms, X, Y)
    assert np.allclose(base[:4], base[0], rtol=1e-12, atol=0)          # 4-fold symmetry
    ms2 = dict(ms, kap0=2.0 * ms["kap0"])
    assert np.allclose(sv2(tr, ms2, X, Y), 2.0 * base, rtol=1e-12)     # Sigma v^2 ~ mass
    tr3 = dict(tr, I0=3.0 * tr["I0"])
    assert np.allclose(sv2(tr3, ms, X, Y), 3.0 * base, rtol=1e-12)     # ~ tracer amplitude
