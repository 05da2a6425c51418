"""Joint log-likelihood of one parameter sample (oracle, FP64).

Eq. chi_general / Eq. Posterior_LD: the joint chi^2 of the terms built here is
chi^2 = chi^2_pix (Eq. chi2 of lens_light over the whole extended image) +
chi^2_dyn (Eq. chi2_dyn) + chi^2_tmd (Eq. chi2_tmd) [+ chi^2_img (Eq. chi2_img) when the
system gives image-position uncertainties], and logL = -chi^2/2 (the Gaussian
normalisation constant is dropped, as chi^2_LD has none).  For a system with a pixelated
source (src_pix = 1, Sect. 3.1.1) the image term is the log-evidence of the source
reconstruction at its optimal regularisation (Eq. evi_ext, oracle/pixsrc.py) in place of
-chi^2_pix / 2, reported as chi2_pix = -2 ln P.

Dynamics chain (Sect. 3.2 and App. A): 1-D MGE of the App. C convergence and of
each lens-light Sersic -> a black-hole Gaussian (sigma_BH, M_BH = f_BH * M_*,
M_* = Upsilon * L_tot, L_tot the total light of the tracer MGE in
convergence units via L_scale) -> deprojection -> JAM on the sub-sampled sky grid
(the cylindrically aligned pair form, or, for systems with jam_align = 1, the
spherically aligned solution of Eqs. J1/J2 by the discrete rule of jam_sph) ->
PSF_kin, binning, v_rms.

An invalid sample (parameter outside its domain, impossible deprojection
cos^2 i >= q'^2 (App. A), or a non-positive deprojected density at the probe
radii, Sect. 3.3) returns logL = -inf and a non-zero status.
"""
import math

import numpy as np

from paper_2504_01302_b300 import synth
from . import cosmo, imaging, jam, jam_sph, kin, lens, lensmodel, mge, pixsrc, tdelay

IDX = synth.IDX

ST_OK, ST_DOMAIN, ST_DEPROJ, ST_NEGDENS, ST_NONFINITE = 0, 1, 2, 3, 4


def check_domain(th, sysd=None):
    """Parameters inside their domain.  Entries a system does not use (lambda_int without a
    sheet; H0 in distance mode 1, D_d and D_dt,int in mode 0) are not checked."""
    sysd = sysd or {}
    g = th[IDX["gamma"]]
    q = th[IDX["q"]]
    inc = th[IDX["inc"]]
    mode1 = int(sysd.get("distance_mode", 0)) == 1
    used = [i for i in range(synth.N_THETA)
            if not (i == IDX["lam_int"] and int(sysd.get("sheet", 0)) == 0)
            and not (i == IDX["H0"] and mode1)
            and not (i in (IDX["D_d"], IDX["D_dt_int"]) and not mode1)]
    if lensmodel.is_composite(sysd):
        # composite class: kappa_s >= 0, r_s > 0, q of the halo in (0, 1], first Chameleon
        # I0 > 0 and w_t > w_c
        mass_ok = (th[0] >= 0 and th[1] > 0 and 0.0 < q <= 1.0 and th[13] > 0
                   and th[14] > float(sysd["ll_wc"]))
    else:
        mass_ok = (th[IDX["theta_E"]] > 0 and 1.0 < g < 3.0 and 0.0 < q <= 1.0
                   and th[IDX["R_e_ll"]] > 0 and th[IDX["I_e_ll"]] > 0)
    ok = (np.all(np.isfinite(th[used])) and mass_ok
          and th[IDX["R_e_src"]] > 0 and th[IDX["n_src"]] > 0
          and 0.0 < inc <= math.pi / 2 + 1e-12 and th[IDX["beta"]] < 1.0
          and th[IDX["upsilon"]] >= 0 and th[IDX["f_bh"]] >= 0
          and (mode1 or th[IDX["H0"]] > 0)
          and (int(sysd.get("sheet", 0)) == 0 or th[IDX["lam_int"]] > 0)
          and (not mode1 or (th[IDX["D_d"]] > 0 and th[IDX["D_dt_int"]] > 0)))
    return bool(ok)


def light_mge(th, sysd):
    """Tracer MGE: one 1-D MGE per lens-light Sersic (Chameleon in the composite class), all
    sharing centre and PA."""
    if lensmodel.is_composite(sysd):
        parts = lensmodel.chameleon_mges(th, sysd)
        return dict(I0=np.concatenate([A for A, _, _ in parts]),
                    sig=np.concatenate([sg for _, sg, _ in parts]),
                    qp=np.concatenate([np.full(len(sg), q) for _, sg, q in parts]))
    P = sysd["mge_P"]
    comps = [(th[IDX["I_e_ll"]], th[IDX["R_e_ll"]], sysd["ll_n"], sysd["ll_q"])]
    comps += [tuple(r) for r in np.asarray(sysd["ll2"]).reshape(-1, 4)]
    I0, sig, qp = [], [], []
    for (I_e, R_e, n, q), N in zip(comps, sysd["n_mge_light"]):
        s, A = mge.mge_1d(mge.sersic_profile(I_e, R_e, n), sysd["light_rmin"],
                          sysd["light_rmax"], N, P)
        I0.append(A)
        sig.append(s)
        qp.append(np.full(N, q))
    return dict(I0=np.concatenate(I0), sig=np.concatenate(sig), qp=np.concatenate(qp))


def mass_mge(th, sysd, L_tot, tr=None):
    """Mass Gaussians of the class (galaxy scaled by lambda_int, then the sheet's, the black hole
    last).  EPL class: the 1-D MGE of the App. C convergence.  Composite class (Sect. 3.3):
    Upsilon_* L_scale times the tracer Gaussians (the lens light), then the halo's."""
    if lensmodel.is_composite(sysd):
        ups = th[IDX["upsilon"]] * sysd["L_scale"]
        Ah, sh_, qh = lensmodel.enfw_mass_mge(th, sysd)
        A = np.concatenate([ups * tr["I0"], Ah])
        s = np.concatenate([tr["sig"], sh_])
        qp = np.concatenate([tr["qp"], qh])
    else:
        s, A = mge.mge_1d(mge.epl_profile(th[IDX["theta_E"]], th[IDX["gamma"]], th[IDX["q"]],
                                          sysd["r_soft"]),
                          sysd["mass_rmin"], sysd["mass_rmax"], sysd["n_mge_mass"], sysd["mge_P"])
        qp = np.full(len(s), th[IDX["q"]])
    # the internal mass sheet (Sect. 3.3, Eq. kappa int): the galaxy (with its black hole)
    # scaled by lambda_int, the sheet's own round Gaussians after it, the black hole last
    lam = lensmodel.lam_of(th, sysd)
    A = lam * A
    sh = lensmodel.sheet_mass(th, sysd)
    if sh is not None:
        A = np.concatenate([A, sh["kap0"]])
        s = np.concatenate([s, sh["sig"]])
        qp = np.concatenate([qp, sh["qp"]])
    if sysd["has_bh"]:
        m_star = th[IDX["upsilon"]] * L_tot * sysd["L_scale"]
        m_bh = th[IDX["f_bh"]] * m_star
        sb = sysd["bh_sigma"]
        A = np.append(A, lam * m_bh / (2 * math.pi * sb * sb))
        s = np.append(s, sb)
        qp = np.append(qp, 1.0)
    return dict(kap0=A, sig=s, qp=qp)


def positive_density(tr, ms, inc):
    """Deprojected mass and tracer densities are positive on probe points
    (R = sigma_n in the equatorial plane and z = q sigma_n on the axis)."""
    for G, key in ((ms, "kap0"), (tr, "I0")):
        rho0, q = jam.deproject(G[key], G["sig"], G["qp"], inc)
        for s in G["sig"]:
            if np.sum(rho0 * np.exp(-s * s / (2 * G["sig"] ** 2))) <= 0:
                return False
            if np.sum(rho0 * np.exp(-s * s / (2 * G["sig"] ** 2 * q * q))) <= 0:
                return False
    return True


def sky_geometry(sysd):
    X, Y = kin.sky_subsamples(sysd["kx"], sysd["ky"], sysd["kss"], sysd["kpix"])
    return X, Y, float(np.max(np.hypot(X, Y)))


def dynamics_setup(th, sysd):
    """Steps of the dynamics chain up to the pair table: (status, pieces)."""
    inc = th[IDX["inc"]]
    tr = light_mge(th, sysd)
    L_tot = float(np.sum(2 * math.pi * tr["I0"] * tr["sig"] ** 2 * tr["qp"]))
    ms = mass_mge(th, sysd, L_tot, tr)
    qmin = min(np.min(tr["qp"]), np.min(ms["qp"]))
    if math.cos(inc) ** 2 >= qmin ** 2:
        return ST_DEPROJ, None
    if not positive_density(tr, ms, inc):
        return ST_NEGDENS, None
    v2u = lensmodel.v2_unit(th, sysd)
    X, Y, r_max = sky_geometry(sysd)
    xp, yp = lens.frame(X, Y, th[IDX["x_c"]], th[IDX["y_c"]], th[IDX["phi"]])
    d = dict(tr=tr, ms=ms, v2u=v2u, r_max=r_max, X=X, xp=xp, yp=yp)
    if sysd.get("jam_align", 0) == 1:
        m = jam_sph.SphModel(tr, ms, inc, th[IDX["beta"]], v2u)
        rule = sph_rule(sysd, tr["sig"], ms["sig"])
        d.update(sph=(m, rule, jam_sph.grid_moments(m, rule)))
    else:
        d.update(tab=jam.table(tr, ms, inc, th[IDX["beta"]], v2u, r_max, sysd["n_gl"]))
    return ST_OK, d


def sph_rule(sysd, sig_light, sig_mass):
    """Discrete rule of the spherically aligned model for this system."""
    dn = jam_sph.DEFAULT_RULE
    return jam_sph.SphRule(sig_light, sig_mass, sysd["kpix"] / sysd["kss"],
                           int(sysd.get("sph_nr", 0) or dn[0]), int(sysd.get("sph_nw", 0) or dn[1]),
                           int(sysd.get("sph_nlos", 0) or dn[2]), sysd["n_gl"])


def sigma_v2(d, xp, yp, chunk=2048):
    """Sigma v_los^2 at galaxy-frame sky points for the system's alignment."""
    if "sph" in d:
        m, rule, grids = d["sph"]
        return jam_sph.sigma_v2_sph(xp, yp, m, rule, grids)
    return jam.sigma_v2_fast(xp, yp, d["tab"], chunk=chunk)


def dynamics(th, sysd, want_maps=False):
    """v_rms per bin (and intermediate maps).  Returns (v_pre, status, extra)."""
    st, d = dynamics_setup(th, sysd)
    if st != ST_OK:
        return None, st, {}
    xp, yp, tr = d["xp"], d["yp"], d["tr"]
    sv2 = sigma_v2(d, xp, yp).reshape(d["X"].shape)
    sb = jam.surface_brightness(xp, yp, tr)
    num, den = kin.bin_moments(sv2, sb, sysd)
    v = np.sqrt(num / den)
    extra = dict(tr=tr, ms=d["ms"], v2u=d["v2u"], r_max=d["r_max"], num=num, den=den)
    if want_maps:
        extra.update(sv2=sv2, sb=sb, xp=xp, yp=yp, tab=d.get("tab"), sph=d.get("sph"))
    return v, ST_OK, extra


def vrms_bins(th, sysd, which, chunk=64):
    """v_rms of the bins listed in ``which`` only (for grids whose full maps are out of
    reach): the same chain as dynamics(), with Sigma v_los^2 and the tracer surface
    brightness evaluated only on the sub-samples that PSF_kin carries into those bins
    (the bins' sub-samples dilated by the kernel half-width) and zero elsewhere.  The
    convolved maps on the bins' own sub-samples, and so their bin sums, are unchanged.
    Returns (v[len(which)], status)."""
    from scipy.ndimage import maximum_filter
    st, d = dynamics_setup(th, sysd)
    if st != ST_OK:
        return None, st
    lab = kin.subsample_bins(sysd["bins"], sysd["kss"])
    K = np.asarray(sysd["kpsf"]).shape[0]
    sup = maximum_filter(np.isin(lab, list(which)).astype(np.uint8), size=K, mode="constant") > 0
    sv2 = np.zeros(lab.shape)
    sb = np.zeros(lab.shape)
    sv2[sup] = sigma_v2(d, d["xp"][sup], d["yp"][sup], chunk=chunk)
    sb[sup] = jam.surface_brightness(d["xp"][sup], d["yp"][sup], d["tr"])
    num, den = kin.bin_moments(sv2, sb, sysd)
    return np.sqrt(num[list(which)] / den[list(which)]), ST_OK


def evaluate(th, sysd, want=False):
    """Full evaluation: dict with logL, the three chi^2 terms, image, v_rms, delays, status."""
    th = np.asarray(th, np.float64)
    out = dict(logL=-np.inf, chi2_pix=np.nan, chi2_dyn=np.nan, chi2_tmd=np.nan, status=ST_OK)
    if not check_domain(th, sysd):
        out["status"] = ST_DOMAIN
        return out
    v, st, extra = dynamics(th, sysd, want_maps=want)
    if st != ST_OK:
        out["status"] = st
        return out
    if sysd.get("src_pix", 0):
        # pixelated source (Sect. 3.1.1): the evidence takes the place of -chi^2_pix / 2
        lnP, lam, s_mp = pixsrc.evidence_term(th, sysd)
        img, c_pix = None, -2.0 * lnP
    else:
        img = imaging.model_image(th, sysd)
        c_pix = imaging.chi2_pix(img, sysd)
    dt = tdelay.delays(th, sysd)
    c_dyn = kin.chi2_dyn(v, sysd)
    c_tmd = tdelay.chi2_tmd(dt, sysd)
    # image positions (Eq. chi2_img) when the system gives their uncertainties
    c_img = tdelay.chi2_img(th, sysd) if sysd.get("img_sig") is not None else 0.0
    logL = -0.5 * (c_pix + c_dyn + c_tmd + c_img)
    if not np.isfinite(logL):
        out["status"] = ST_NONFINITE
        return out
    out.update(logL=logL, chi2_pix=c_pix, chi2_dyn=c_dyn, chi2_tmd=c_tmd, chi2_img=c_img, image=img,
               vrms=v, delays=dt, extra=extra)
    if sysd.get("src_pix", 0):
        out.update(lnP=lnP, lam=lam, s_mp=s_mp)
    return out


def loglike(th, sysd):
    return evaluate(th, sysd)["logL"]


def used_params(sysd):
    """Indices of the parameter entries a system uses: lambda_int only with a sheet, H0 only in
    distance mode 0, D_d and D_dt,int only in mode 1 (the others do not enter logL)."""
    mode1 = int(sysd.get("distance_mode", 0)) == 1
    out = [i for i in range(synth.N_BASE) if not (mode1 and i == IDX["H0"])]
    if int(sysd.get("sheet", 0)):
        out.append(IDX["lam_int"])
    if mode1:
        out += [IDX["D_d"], IDX["D_dt_int"]]
    return out


def grad_fd(th, sysd, h_rel=1e-6, which=None):
    """Central finite differences of logL with h = h_rel * parameter scale (FP64), over the
    parameters the system uses (or those in which); the others are 0."""
    th = np.asarray(th, np.float64)
    g = np.zeros(len(th))
    idx = used_params(sysd) if which is None else which
    for i in idx:
        h = h_rel * synth.THETA_SCALE[i]
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        g[i] = (loglike(tp, sysd) - loglike(tm, sysd)) / (2 * h)
    return g


# ---------------------------------------------------------------------------
# mock systems: data = oracle model at the truth + seeded noise
# ---------------------------------------------------------------------------

def build_system(base, theta_true, noise):
    """Fill data, kinematics and delays of a fixed system from the oracle model."""
    s = dict(base)
    s["data"] = np.zeros((s["ny"], s["nx"]), np.float32)
    s["v_obs"] = np.ones(s["n_bins"], np.float32)
    s["v_sig"] = np.ones(s["n_bins"], np.float32)
    # quasar images: Newton solution of the lens equation for the quasar source point
    guesses = synth.ring_images(1.65 if lensmodel.is_composite(s) else theta_true[IDX["theta_E"]],
                                s["qso_beta"])
    img = lensmodel.solve_images(s["qso_beta"], theta_true, s, guesses)
    s["img_xy"] = img
    s["dt_obs"] = np.zeros(len(img) - 1)
    s["dt_sig"] = np.ones(len(img) - 1)
    # the data come from the Sersic source; a pixelated-source system then fits them
    ev = evaluate(theta_true, dict(s, src_pix=0))
    assert ev["status"] == ST_OK, ev["status"]
    m = ev["image"]
    s["data"] = (m + np.asarray(s["sigma"], np.float64) * noise["img"]).astype(np.float32)
    v = ev["vrms"]
    s["v_sig"] = (0.02 * v).astype(np.float32)
    s["v_obs"] = (v + 0.02 * v * noise["kin"]).astype(np.float32)
    dt = ev["delays"]
    sig = 0.016 * np.abs(dt) + 0.1
    s["dt_sig"] = sig
    s["dt_obs"] = dt + sig * noise["dt"][:len(dt)]
    return s


def workload(w, small=False):
    """Mock systems, parameter samples and system ids of workload w."""
    bases, B = synth.workload_systems(w)
    systems = []
    for si, b in enumerate(bases):
        truth = synth.theta_truth_composite() if lensmodel.is_composite(b) else synth.theta_truth(0 if w == 0 else 1)
        systems.append(build_system(b, truth, synth.noise_draws(b, 1000 * w + si + 500)))
    th, sid = synth.workload_thetas(w, B, len(systems))
    return systems, th, sid
