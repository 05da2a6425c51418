"""Mock systems for the tests: seeded geometry (synth) + oracle data at the truth."""
import functools

import numpy as np

from oracle import model
from paper_2504_01302_b300 import synth


def small_base(seed=7, n_px=48, ss=2, psf_k=7, sky=20, kss=2, n_mass=8, n_light=(5, 4), n_gl=16,
               n_bins=12, has_bh=True, n_sis=1, second_light=True):
    """A small system with every model feature (EPL, shear, SIS, BH, two lens lights),
    sized so that every kernel runs several tiles with a ragged last one."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return synth.base_system(f"small{seed}", n_img_px=n_px, ss=ss, psf_k=psf_k, sky=sky, kss=kss,
                             n_mass=n_mass, n_light=list(n_light) if second_light else [n_light[0]],
                             n_gl=n_gl, n_bins=n_bins, bins="voronoi", rng=rng, has_bh=has_bh,
                             n_sis=n_sis, second_light=second_light)


@functools.lru_cache(maxsize=None)
def small_system(seed=7, **kw):
    b = small_base(seed, **dict(kw))
    return model.build_system(b, synth.theta_truth(1), synth.noise_draws(b, 9000 + seed))


@functools.lru_cache(maxsize=None)
def workload(w):
    return model.workload(w)


def prior_thetas(n, seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    return synth.draw_prior(rng, n)


def near_truth_thetas(n, seed=13, scale=0.002):
    """Draws close to the truth (the posterior region a sampler spends its time in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    span = synth.PRIOR_HI - synth.PRIOR_LO
    th = synth.theta_truth(1)[None, :] + scale * span * rng.standard_normal((n, synth.N_THETA))
    th[:, synth.IDX["f_bh"]] = np.abs(th[:, synth.IDX["f_bh"]])
    th[:, synth.IDX["inc"]] = np.minimum(th[:, synth.IDX["inc"]], np.pi / 2)
    return th


def logl_tol(ref):
    """|logL_gpu - logL_oracle| bound: 0.05 absolute (the workload's bar, met near the
    posterior) plus 5e-6 |logL|.  FP32 ray shooting leaves ~1e-7 arcsec in beta; the
    source's logarithmic gradient (up to ~20/arcsec) turns that into model errors up
    to ~2e-6 relative, coherent over the arcs, so far from the data (chi^2 >> N) the
    chi^2 error grows like 2 * 2e-6 * chi^2."""
    return 0.05 + 5e-6 * abs(ref)


@functools.lru_cache(maxsize=None)
def ifu_system():
    """The IFU-scale system (400^2 x 3 image, 31^2 PSF, EPL + shear + 2 SIS, 40 + 2 x 20 MGE
    + BH, 128^2 x 4 sky, 400 bins, GL64) with imaging data and delays from the oracle at the
    truth.  The oracle's full v_rms map is out of reach at this size (2.75e10 integrand
    evaluations), so v_obs is a seeded draw around 300 km/s with 2 % errors: the parity
    checks compare the two paths on the same data, not the fit."""
    from oracle import imaging, lens, tdelay
    bases, _ = synth.workload_systems(4)
    s = dict(bases[0])
    truth = synth.theta_truth(1)
    nz = synth.noise_draws(s, 4500)
    s["img_xy"] = lens.solve_images(s["qso_beta"], truth, s["sis"],
                                    synth.ring_images(truth[synth.IDX["theta_E"]], s["qso_beta"]))
    m = imaging.model_image(truth, s)
    s["data"] = (m + np.asarray(s["sigma"], np.float64) * nz["img"]).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(4501))
    v = 300.0 * (1.0 + 0.05 * rng.standard_normal(s["n_bins"]))
    s["v_obs"] = v.astype(np.float32)
    s["v_sig"] = (0.02 * v).astype(np.float32)
    s["dt_obs"] = np.zeros(len(s["img_xy"]) - 1)
    s["dt_sig"] = np.ones(len(s["img_xy"]) - 1)
    dt = tdelay.delays(truth, s)
    sig = 0.016 * np.abs(dt) + 0.1
    s["dt_sig"] = sig
    s["dt_obs"] = dt + sig * nz["dt"][:len(dt)]
    return s
