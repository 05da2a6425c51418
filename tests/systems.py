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
    chi^2 error grows like 2 * 2e-6 * chi^2 (derivation in the design doc)."""
    return 0.05 + 5e-6 * abs(ref)
