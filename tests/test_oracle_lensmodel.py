"""Pins of the mass classes' lens model, sheet and distance modes (oracle/lensmodel.py),
Sect. 3.3 and Sect. 2.2-2.3: the sheet's Jacobian and the class's psi <-> alpha <-> Jacobian by
central differences; the ideal sheet as the exact mass-sheet transform of the delays
(Fermat-potential differences scale by lambda, Eq. transformed MST) and of the mapped-back
image positions; distance mode 1 at the distances of an H0 reproducing mode 0 (Eqs.
critical_sfd, sfd final); v_rms of the class linear in lambda through its mass Gaussians; a
sheet with lambda > 1 turning the outer density negative, which the model rejects (Sect. 3.3:
negative convergence is rejected by JAM)."""
import numpy as np
import pytest

from oracle import cosmo, jam, lensmodel, mass_sheet, model, tdelay
from paper_2504_01302_b300 import synth

from . import systems

I = synth.IDX


def test_sheet_jacobian_by_differences():
    # the sheet varies on the 45" core scale: a wide step keeps the differences of its
    # deflection (whose plain form cancels about three digits) far above rounding
    h = 1e-3
    for lam in (0.7, 1.3):
        sh = dict(lam=lam, kind="dpie", rc=45.0, rt=45.09)
        for x, y in ((0.3, -0.2), (1.7, 0.9), (-12.0, 30.0)):
            A = lambda a, b: np.array(mass_sheet.sheet_alpha(np.array([a]), np.array([b]), sh))[:, 0]
            J = lensmodel.sheet_jac(np.array([x]), np.array([y]), sh)
            dx = (A(x + h, y) - A(x - h, y)) / (2 * h)
            dy = (A(x, y + h) - A(x, y - h)) / (2 * h)
            ref = np.array([dx[0], dy[0], dx[1], dy[1]])
            got = np.array([J[0][0], J[1][0], J[2][0], J[3][0]])
            assert np.max(np.abs(got - ref)) < 1e-8 * max(1.0, np.max(np.abs(ref))), (x, y, got, ref)


@pytest.mark.parametrize("lam,kind", [(0.85, 1), (1.2, 1), (0.8, 2)])
def test_class_potential_deflection_jacobian(lam, kind):
    s = dict(systems.small_system(7), sheet=kind)
    th = synth.theta_truth(1).copy()
    th[I["lam_int"]] = lam
    h = 1e-5
    for x, y in ((0.9, -1.2), (-1.4, 0.6)):
        P = lambda a, b: lensmodel.psi(np.array([a]), np.array([b]), th, s)[0]
        A = lambda a, b: np.array(lensmodel.alpha(np.array([a]), np.array([b]), th, s))[:, 0]
        ax, ay = A(x, y)
        assert abs((P(x + h, y) - P(x - h, y)) / (2 * h) - ax) < 1e-7
        assert abs((P(x, y + h) - P(x, y - h)) / (2 * h) - ay) < 1e-7
        J = lensmodel.jac(np.array([x]), np.array([y]), th, s)
        dx = (A(x + h, y) - A(x - h, y)) / (2 * h)
        dy = (A(x, y + h) - A(x, y - h)) / (2 * h)
        assert np.allclose([J[0][0], J[1][0], J[2][0], J[3][0]], [dx[0], dy[0], dx[1], dy[1]],
                           atol=1e-7)


def test_ideal_sheet_is_the_mass_sheet_transform_of_delays_and_images():
    s0 = dict(systems.small_system(7))
    s0["img_sig"] = np.full(len(s0["img_xy"]), 0.003)
    th = systems.near_truth_thetas(1, seed=5)[0]
    d0 = tdelay.delays(th, s0)
    pre0 = tdelay.predicted_images(th, s0)
    for lam in (0.8, 1.25):
        s = dict(s0, sheet=2)
        t = th.copy()
        t[I["lam_int"]] = lam
        assert np.allclose(tdelay.delays(t, s), lam * d0, rtol=1e-9, atol=1e-12)
        assert np.max(np.abs(tdelay.predicted_images(t, s) - pre0)) < 1e-9


def test_distance_mode_1_reproduces_mode_0():
    s0 = systems.small_system(7)
    th = systems.near_truth_thetas(1, seed=6)[0]
    H0 = th[I["H0"]]
    D_d, _, _, D_dt = cosmo.distances(s0["z_d"], s0["z_s"], H0, s0["omega_m"])
    s1 = dict(s0, distance_mode=1)
    t1 = th.copy()
    t1[I["D_d"]] = D_d
    t1[I["D_dt_int"]] = (1 - s0["kappa_ext"]) * D_dt
    t1[I["H0"]] = np.nan  # not used in mode 1
    e0, e1 = model.evaluate(th, s0), model.evaluate(t1, s1)
    assert e1["status"] == 0
    assert np.allclose(e1["delays"], e0["delays"], rtol=1e-12)
    assert np.allclose(e1["vrms"], e0["vrms"], rtol=1e-12)
    # v_rms depends on D_dt,int / D_d only (Eq. sfd final): doubling both leaves it unchanged,
    # raising D_dt,int alone by 4 doubles it
    t2 = t1.copy()
    t2[I["D_d"]] *= 2
    t2[I["D_dt_int"]] *= 2
    assert np.allclose(model.evaluate(t2, s1)["vrms"], e1["vrms"], rtol=1e-12)
    t3 = t1.copy()
    t3[I["D_dt_int"]] *= 4
    assert np.allclose(model.evaluate(t3, s1)["vrms"], 2 * e1["vrms"], rtol=1e-12)


def test_class_mass_is_lambda_galaxy_plus_sheet():
    """Sigma v^2 is linear in the mass Gaussians (pinned in test_oracle_mass_sheet), so the
    class's mass model must be lambda x (galaxy + black hole) followed by the sheet's own
    Gaussians."""
    s0 = systems.small_system(7)
    s = dict(s0, sheet=1)
    th = systems.near_truth_thetas(1, seed=8)[0]
    th[I["lam_int"]] = 0.9
    tr = model.light_mge(th, s)
    L = float(np.sum(2 * np.pi * tr["I0"] * tr["sig"] ** 2 * tr["qp"]))
    ms0 = model.mass_mge(th, s0, L)
    ms = model.mass_mge(th, s, L)
    ref = mass_sheet.class_mass(dict(kap0=ms0["kap0"][:-1], sig=ms0["sig"][:-1], qp=ms0["qp"][:-1]),
                                0.9, n=40, P=s["mge_P"], rmin=0.1, rmax=1000.0)
    n = len(ref["kap0"])
    assert np.allclose(ms["kap0"][:n], ref["kap0"], rtol=1e-14)
    assert np.allclose(ms["sig"][:n], ref["sig"], rtol=1e-14)
    assert abs(ms["kap0"][-1] - 0.9 * ms0["kap0"][-1]) <= 1e-14 * abs(ms0["kap0"][-1])


def test_sheet_above_one_gives_negative_density():
    s = dict(systems.small_system(7), sheet=1)
    th = systems.near_truth_thetas(1, seed=9)[0]
    for lam, st in ((0.8, model.ST_OK), (1.0, model.ST_OK), (1.3, model.ST_NEGDENS)):
        t = th.copy()
        t[I["lam_int"]] = lam
        ev = model.evaluate(t, s)
        assert ev["status"] == st, (lam, ev["status"])
        if st != model.ST_OK:
            assert ev["logL"] == -np.inf
