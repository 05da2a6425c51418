"""Seeded synthetic inputs for the joint lensing + dynamics likelihood.

This module holds NO arithmetic of the likelihood itself.  It builds the
fixed, parameter-independent pieces of a mock system -- grid sizes, sampled
Gaussian PSFs, kinematic bin maps, parameter vectors drawn from the priors,
unit-normal noise draws -- with NumPy ``PCG64`` generators seeded per workload
(seed 1000 + workload index, per-system sub-seeds 1000*w + s).

The shapes follow the paper's RXJ1131 set-up: HST ACS 0.05"/px imaging with a
0.1" FWHM PSF, a +-1" kinematic field of view with a 0.14" FWHM kinematic PSF
(Sect. 4), 2 % kinematic errors (Eq. idea data), 1.6 % time-delay errors
(Sect. 1), lens at z=0.295 and source at z=0.654 with H0=82.5, Om=0.27
(Table 2).  The paper's real data (HST imaging, COSMOGRAIL delays, JWST IFU
kinematics) are not available; these seeded inputs stand in for them.

Noise-free model values (the mock data themselves) are NOT produced here:
whoever builds a full system fills ``data``, ``v_obs`` and ``dt_obs`` from a
model evaluated at ``theta_true`` plus the unit-normal draws returned here.
"""
from __future__ import annotations

import math

import numpy as np

# Parameter vector layout (23 values, float64).  Angles are in radians.  The last three are
# the internal mass sheet's lambda_int (used by systems with a sheet) and the lens and model
# time-delay distances D_d, D_dt,int [Mpc] (used by systems in distance mode 1, which then
# ignore H0).
THETA_NAMES = (
    "theta_E", "gamma", "q", "phi", "x_c", "y_c", "gamma_ext", "phi_ext",
    "I_e_src", "R_e_src", "n_src", "x_src", "y_src", "I_e_ll", "R_e_ll",
    "inc", "beta", "upsilon", "f_bh", "H0", "lam_int", "D_d", "D_dt_int",
)
N_BASE = 20  # entries drawn by draw_prior (the others stay at their Table 2 mock values)
N_THETA = len(THETA_NAMES)
IDX = {n: i for i, n in enumerate(THETA_NAMES)}

# Scale of each parameter, used to size finite-difference steps (h = 1e-6 * scale).
THETA_SCALE = np.array([
    1.0, 1.0, 1.0, 1.0, 0.1, 0.1, 0.1, 1.0,
    1.0, 0.1, 1.0, 0.1, 0.1, 1.0, 1.0,
    1.0, 0.1, 1.0, 0.01, 100.0, 1.0, 100.0, 100.0,
])

DEG = math.pi / 180.0
FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def sampled_gaussian_psf(k: int, fwhm_pix: float) -> np.ndarray:
    """k x k Gaussian sampled at pixel centres, normalised to unit sum (float32)."""
    assert k % 2 == 1
    s = fwhm_pix * FWHM_TO_SIGMA
    h = (k - 1) // 2
    ax = np.arange(-h, h + 1, dtype=np.float64)
    g = np.exp(-0.5 * (ax[:, None] ** 2 + ax[None, :] ** 2) / (s * s))
    g /= g.sum()
    return g.astype(np.float32)


def truncated_gaussian_psf(fwhm_pix: float, nsig: float = 3.0) -> np.ndarray:
    """Gaussian sampled on the kinematic sub-grid, truncated at nsig sigma, unit sum."""
    s = fwhm_pix * FWHM_TO_SIGMA
    h = max(1, int(math.floor(nsig * s)))
    ax = np.arange(-h, h + 1, dtype=np.float64)
    g = np.exp(-0.5 * (ax[:, None] ** 2 + ax[None, :] ** 2) / (s * s))
    g[(ax[:, None] ** 2 + ax[None, :] ** 2) > (nsig * s) ** 2 + 1e-9] = 0.0
    g /= g.sum()
    return g.astype(np.float32)


def spaxel_centres(kx: int, ky: int, kpix: float):
    x = (np.arange(kx) - 0.5 * (kx - 1)) * kpix
    y = (np.arange(ky) - 0.5 * (ky - 1)) * kpix
    return np.meshgrid(x, y)


def safe_margin_spaxels(kpsf: np.ndarray, kss: int) -> int:
    """Spaxels to leave unbinned at each grid edge so that no binned sub-sample
    is nearer the edge than the kinematic PSF radius."""
    h = (kpsf.shape[0] - 1) // 2
    return int(math.ceil(h / kss))


def annular_bins(kx, ky, kpix, n_bins, r_out, margin):
    """Equal-width circular annuli out to r_out (inside the PSF-safe interior)."""
    X, Y = spaxel_centres(kx, ky, kpix)
    r = np.hypot(X, Y)
    b = np.floor(r / r_out * n_bins).astype(np.int32)
    b[r >= r_out] = -1
    inner = np.zeros((ky, kx), bool)
    inner[margin:ky - margin, margin:kx - margin] = True
    b[~inner] = -1
    # renumber the non-empty annuli consecutively (the innermost may hold no spaxel centre)
    used = np.unique(b[b >= 0])
    remap = -np.ones(n_bins, np.int32)
    remap[used] = np.arange(len(used), dtype=np.int32)
    return np.where(b >= 0, remap[np.maximum(b, 0)], -1).astype(np.int32)


def voronoi_like_bins(rng, kx, ky, kpix, n_bins, margin):
    """Nearest-generator assignment of the PSF-safe interior spaxels to n_bins
    seeded generators (ties to the lower index).  Generators are drawn with a
    density rising towards the centre, like S/N-driven Voronoi bins; empty bins
    are re-seeded on an unused spaxel until every bin holds a spaxel."""
    X, Y = spaxel_centres(kx, ky, kpix)
    inner = np.zeros((ky, kx), bool)
    inner[margin:ky - margin, margin:kx - margin] = True
    pts = np.stack([X[inner], Y[inner]], 1)
    half = min(X[inner].max(), Y[inner].max())
    # radius ~ half * u^1.5 concentrates generators near the centre
    u = rng.random(n_bins)
    ang = rng.random(n_bins) * 2 * math.pi
    rad = half * u ** 1.5
    gen = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    for _ in range(100):
        d2 = ((pts[:, None, :] - gen[None, :, :]) ** 2).sum(-1)
        lab = np.argmin(d2, axis=1)
        counts = np.bincount(lab, minlength=n_bins)
        empty = np.nonzero(counts == 0)[0]
        if len(empty) == 0:
            break
        for e in empty:
            gen[e] = pts[rng.integers(len(pts))] + 1e-6 * (e + 1)
    b = -np.ones((ky, kx), np.int32)
    b[inner] = lab.astype(np.int32)
    return b


def base_system(name: str, *, n_img_px: int, ss: int, psf_k: int, sky: int, kss: int,
                n_mass: int, n_light, n_gl: int, n_bins: int, bins: str, rng,
                has_bh: bool, n_sis: int, second_light: bool) -> dict:
    """Fixed (parameter-independent) part of one mock system."""
    pix = 0.05
    psf = sampled_gaussian_psf(psf_k, 0.1 / pix)
    kpix = 2.0 / sky                              # +-1" field of view
    kpsf = truncated_gaussian_psf(0.14 / (kpix / kss))
    margin = safe_margin_spaxels(kpsf, kss)
    if bins == "annular":
        b = annular_bins(sky, sky, kpix, n_bins, 0.8, margin)
    else:
        b = voronoi_like_bins(rng, sky, sky, kpix, n_bins, margin)
    h = (psf_k - 1) // 2
    mask = np.zeros((n_img_px, n_img_px), np.uint8)
    mask[h:n_img_px - h, h:n_img_px - h] = 1
    sis = np.array([[0.2, -0.3, 0.6], [0.1, 0.8, -0.9]], np.float64)[:n_sis]
    ll2 = (np.array([[0.3, 0.3, 1.0, 0.85]], np.float64) if second_light
           else np.zeros((0, 4), np.float64))
    if isinstance(n_light, int):
        n_light = [n_light] + ([n_light] if second_light else [])
    return dict(
        name=name, nx=n_img_px, ny=n_img_px, ss=ss, pix=pix,
        sigma=np.full((n_img_px, n_img_px), 0.01, np.float32), mask=mask, psf=psf,
        src_q=0.9, src_phi=0.0, ll_n=4.0, ll_q=0.85, ll2=ll2, sis=sis, r_soft=0.01,
        kx=sky, ky=sky, kss=kss, kpix=kpix, kpsf=kpsf, bins=b,
        n_bins=int(b.max()) + 1,
        n_mge_mass=n_mass, n_mge_light=list(n_light), mge_P=10, n_gl=n_gl,
        mass_rmin=0.005, mass_rmax=50.0, light_rmin=0.005, light_rmax=20.0,
        has_bh=bool(has_bh), bh_sigma=0.01, L_scale=1.0,
        z_d=0.295, z_s=0.654, omega_m=0.27, kappa_ext=0.0,
        # quasar source point used to place the images (Newton-solved by the model side)
        qso_beta=np.array([0.03, -0.02]),
    )


def theta_truth(workload: int) -> np.ndarray:
    t = np.zeros(N_THETA)
    t[IDX["theta_E"]] = 1.5 if workload == 0 else 1.65
    t[IDX["gamma"]] = 2.0
    t[IDX["q"]] = 0.8
    t[IDX["phi"]] = 30 * DEG
    t[IDX["x_c"]] = 0.0
    t[IDX["y_c"]] = 0.0
    t[IDX["gamma_ext"]] = 0.05 if workload == 0 else 0.09
    t[IDX["phi_ext"]] = 1.42
    t[IDX["I_e_src"]] = 1.0
    t[IDX["R_e_src"]] = 0.2
    t[IDX["n_src"]] = 1.5
    t[IDX["x_src"]] = 0.05
    t[IDX["y_src"]] = 0.02
    t[IDX["I_e_ll"]] = 0.5
    t[IDX["R_e_ll"]] = 1.0
    t[IDX["inc"]] = 60 * DEG if workload == 0 else 84.3 * DEG
    t[IDX["beta"]] = 0.1 if workload == 0 else 0.15
    t[IDX["upsilon"]] = 1.0 if workload == 0 else 1.95
    t[IDX["f_bh"]] = 0.0 if workload == 0 else 0.0025
    t[IDX["H0"]] = 82.5
    # Table 2 mock values: no sheet (lambda_int = 1), D_d = 775 Mpc, D_dt,int = 1823 Mpc
    t[IDX["lam_int"]] = 1.0
    t[IDX["D_d"]] = 775.0
    t[IDX["D_dt_int"]] = 1823.0
    return t


PRIOR_LO = np.array([1.60, 1.8, 0.7, 25 * DEG, -0.02, -0.02, 0.07, 1.32,
                     0.9, 0.18, 1.35, 0.04, 0.01, 0.45, 0.9,
                     80 * DEG, -0.3, 0.5, 0.0, 50.0, 0.5, 600.0, 1000.0])
PRIOR_HI = np.array([1.70, 2.2, 0.9, 35 * DEG, 0.02, 0.02, 0.11, 1.52,
                     1.1, 0.22, 1.65, 0.06, 0.03, 0.55, 1.1,
                     90 * DEG, 0.3, 3.5, 0.005, 120.0, 1.5, 1000.0, 4000.0])


def draw_prior(rng, B: int) -> np.ndarray:
    """B parameter vectors from the uniform priors around the RXJ1131-like truth
    (inclination, anisotropy, M/L and H0 ranges as in Table 2).  Only the first N_BASE
    entries are drawn; lambda_int, D_d and D_dt,int keep their mock values (1, 775, 1823)."""
    u = rng.random((B, N_BASE))
    th = np.tile(theta_truth(1), (B, 1))
    th[:, :N_BASE] = PRIOR_LO[:N_BASE] + u * (PRIOR_HI[:N_BASE] - PRIOR_LO[:N_BASE])
    return th


# The composite mass class (Sect. 3.3) gives entries 0, 1, 2, 13, 14 other meanings: the
# halo's kappa_s, r_s [arcsec], q (Eq. kappa_enfw; Table 2's rho_s, r_s, q_enfw) and the first
# Chameleon's I0 and w_t [arcsec] (Eq. Chameleon).  Mock truth and prior ranges: kappa_s 0.09
# (with the baryons, a mean convergence near 1 inside 1.65"), r_s 23 (Table 2), q 0.56 (Table
# 2), I0 0.6 and w_t 1.5" (w_c 0.05", q 0.85; a second Chameleon 0.3, 0.3", 3", 0.9 fixed).
COMPOSITE_TRUTH = {0: 0.09, 1: 23.0, 2: 0.56, 13: 0.6, 14: 1.5}
COMPOSITE_PRIOR = {0: (0.07, 0.11), 1: (20.4, 25.6), 2: (0.46, 0.66), 13: (0.54, 0.66),
                   14: (1.35, 1.65)}


def theta_truth_composite() -> np.ndarray:
    t = theta_truth(1)
    for i, v in COMPOSITE_TRUTH.items():
        t[i] = v
    return t


def draw_prior_composite(rng, B: int, lam_hi: float = 1.0) -> np.ndarray:
    """B parameter vectors for the composite class with the sheet in distance mode 1 (the
    entries of draw_prior_sheet, the class's own entries redrawn from COMPOSITE_PRIOR)."""
    th = draw_prior_sheet(rng, B, lam_hi=lam_hi)
    u = rng.random((B, len(COMPOSITE_PRIOR)))
    for n, (i, (lo, hi)) in enumerate(sorted(COMPOSITE_PRIOR.items())):
        th[:, i] = lo + u[:, n] * (hi - lo)
    return th


def composite_light(system: dict) -> dict:
    """Turn a base system into the composite class: Chameleon lens light (first component
    w_c 0.05", q 0.85; a second fixed Chameleon), the halo expanded on the mass range."""
    s = dict(system)
    s.update(mass_class=1, ll_wc=0.05, ll_q=0.85,
             ll2=np.array([[0.3, 0.3, 3.0, 0.9]], np.float64)[:len(np.asarray(system["ll2"]).reshape(-1, 4))])
    return s


def draw_prior_sheet(rng, B: int, lam_hi: float = 1.5) -> np.ndarray:
    """B parameter vectors for systems with the internal mass sheet in distance mode 1: every
    entry drawn, lambda_int in [0.5, lam_hi] (Table 2: [0.5, 1.5]), D_d in [600, 1000] and
    D_dt,int in [1000, 4000] Mpc (Table 2), H0 drawn too but unused."""
    u = rng.random((B, N_THETA))
    hi = PRIOR_HI.copy()
    hi[IDX["lam_int"]] = lam_hi
    return PRIOR_LO + u * (hi - PRIOR_LO)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def arc_mask(n_px: int, pix: float, r_in: float, r_out: float) -> np.ndarray:
    """Pixels whose centres lie in the annulus r_in <= r < r_out around the image centre (the
    arcs that a pixelated source is fitted to)."""
    c = (np.arange(n_px) - 0.5 * (n_px - 1)) * pix
    r = np.hypot(c[None, :], c[:, None])
    return ((r >= r_in) & (r < r_out)).astype(np.uint8)


def workload_systems(w: int, small: bool = False):
    """Fixed parts of the mock systems of workload w (0..4) and the batch size.

    0: single-sample correctness case (64^2, SIE, 10+10 Gaussians, 32^2 sky, GL32, 20 annuli)
    1: RXJ1131-scale forward (200^2 x2, 21^2 PSF, 20+2x10+BH, 60^2 sky x4, GL32, 50 bins), B=256
    2: workload 1's system, B=64, forward + gradient
    3: 8 uneven systems, 1024 samples split multinomially
    4: IFU-scale (400^2 x3, 31^2 PSF, 40+2x20+BH, 128^2 sky x4, GL64, 400 bins), B=4096
    5: workload 1's system with the spherically aligned Jeans model (Eqs. J1/J2; polar
       grid 128 x 8, 32 line-of-sight nodes), B=256
    6: workload 4's system with the spherically aligned Jeans model (same rule), B=4096
    7: workload 1's system as the EPL mass class with the internal mass sheet (the dPIE of
       Eq. dpie_kappa, 40 Gaussians on [0.1, 1000]") and sampled distances D_d, D_dt,int
       (distance mode 1, Table 2), B=256
    8: workload 1's system as the composite mass class (two Chameleons scaled by Upsilon_*,
       the elliptical NFW halo, the black hole) with the dPIE sheet in distance mode 1: the
       paper's own joint model (Sect. 3.3), B=256
    9: workload 1's system with the pixelated source (Sect. 3.1.1): a 30 x 30 grid over
       +-0.6" around the source, fitted to the arcs in the annulus 0.9" - 2.5" (N_d = 6,840
       pixels, N_s = 900: Table 1's O(10^4) and O(10^3)), B=296 (two samples per SM)
    10: Table 3's timing configuration: workload 8's composite system with a 64 x 64 source grid
       over +-0.6" around the source, fitted to the arcs in 0.8" - 2.95" (N_d = 10,148,
       N_s = 4,096), one sample per call (B=1)
    """
    rng = np.random.Generator(np.random.PCG64(1000 + {5: 1, 6: 4, 7: 1, 8: 1, 9: 1, 10: 1}.get(w, w)))
    if w == 0:
        s = base_system("w0", n_img_px=64, ss=1, psf_k=11, sky=32, kss=1, n_mass=10,
                        n_light=10, n_gl=32, n_bins=20, bins="annular", rng=rng,
                        has_bh=False, n_sis=0, second_light=False)
        return [s], 1
    if w in (1, 2, 5, 7, 8, 9, 10):
        s = base_system("w1", n_img_px=200, ss=2, psf_k=21, sky=60, kss=4, n_mass=20,
                        n_light=10, n_gl=32, n_bins=50, bins="voronoi", rng=rng,
                        has_bh=True, n_sis=1, second_light=True)
        if w == 9:
            t = theta_truth(1)
            c = (float(t[IDX["x_src"]]), float(t[IDX["y_src"]]))
            s.update(name="w9", src_pix=1, spx_n=(30, 30),
                     spx_box=(c[0] - 0.6, c[0] + 0.6, c[1] - 0.6, c[1] + 0.6),
                     mask=arc_mask(s["nx"], s["pix"], 0.9, 2.5))
            return [s], 296
        if w == 5:
            s.update(name="w5", jam_align=1, sph_nr=128, sph_nw=8, sph_nlos=32)
        if w == 7:
            s.update(name="w7", sheet=1, distance_mode=1)
        if w in (8, 10):
            s = composite_light(s)
            s.update(name="w8", sheet=1, distance_mode=1)
        if w == 10:
            t = theta_truth_composite()
            c = (float(t[IDX["x_src"]]), float(t[IDX["y_src"]]))
            s.update(name="w10", src_pix=1, spx_n=(64, 64),
                     spx_box=(c[0] - 0.6, c[0] + 0.6, c[1] - 0.6, c[1] + 0.6),
                     mask=arc_mask(s["nx"], s["pix"], 0.8, 2.95))
            return [s], 1
        return [s], (64 if w == 2 else 256)
    if w == 3:
        systems = []
        for si in range(8):
            r = np.random.Generator(np.random.PCG64(1000 * w + si))
            n_px = int(r.integers(64, 257))
            ss = int(r.choice([1, 2, 3]))
            k = int(r.choice([11, 15, 21]))
            nm = int(r.integers(8, 31))
            nl = int(r.integers(8, 31))
            nb = int(r.integers(20, 121))
            ngl = int(r.integers(24, 65))
            sky = int(r.integers(32, 65))
            kss = int(r.choice([2, 4]))
            l1 = max(4, nl // 2)
            s = base_system(f"w3s{si}", n_img_px=n_px, ss=ss, psf_k=k, sky=sky, kss=kss,
                            n_mass=nm, n_light=[l1, max(4, nl - l1)], n_gl=ngl, n_bins=nb,
                            bins="voronoi", rng=r, has_bh=True, n_sis=1, second_light=True)
            systems.append(s)
        return systems, 1024
    if w in (4, 6):
        s = base_system("w4", n_img_px=400, ss=3, psf_k=31, sky=128, kss=4, n_mass=40,
                        n_light=20, n_gl=64, n_bins=400, bins="voronoi", rng=rng,
                        has_bh=True, n_sis=2, second_light=True)
        if w == 6:
            s.update(name="w6", jam_align=1, sph_nr=128, sph_nw=8, sph_nlos=32)
        return [s], 4096
    raise ValueError(w)


def workload_thetas(w: int, B: int, n_sys: int):
    """Parameter samples and their system ids for workload w."""
    rng = np.random.Generator(np.random.PCG64(1000 + w + 77))
    if w == 0:
        return theta_truth(0)[None, :].copy(), np.zeros(1, np.int32)
    # the sheet workload draws lambda_int in [0.5, 1]: above 1 the EPL class's outer density
    # turns negative and the Jeans model rejects the sample (Sect. 3.3)
    if w == 7:
        th = draw_prior_sheet(rng, B, lam_hi=1.0)
    elif w == 8:
        th = draw_prior_composite(rng, B)
    elif w == 10:
        # the timing configuration's sample: the mock's own parameters (the regularisation
        # search then ends inside its interval, as near a posterior mode)
        th = np.tile(theta_truth_composite(), (B, 1))
    else:
        th = draw_prior(rng, B)
    if n_sys == 1:
        sid = np.zeros(B, np.int32)
    else:
        counts = rng.multinomial(B, np.full(n_sys, 1.0 / n_sys))
        sid = np.repeat(np.arange(n_sys, dtype=np.int32), counts)
        rng.shuffle(sid)
    return th, sid


def noise_draws(system: dict, seed: int) -> dict:
    """Unit-normal draws for the image, the kinematic bins and the delays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return dict(
        img=rng.standard_normal((system["ny"], system["nx"])),
        kin=rng.standard_normal(system["n_bins"]),
        dt=rng.standard_normal(8),
    )


def ring_images(theta_E: float, beta, n_img: int = 4) -> np.ndarray:
    """Rough quasar image positions on the Einstein ring (used only where an exact
    lens-equation solution is not needed, e.g. timing runs)."""
    ang = np.array([0.35, 1.9, 3.5, 5.0])[:n_img]
    r = theta_E * (1 + 0.05 * np.cos(ang))
    return np.stack([r * np.cos(ang) + beta[0], r * np.sin(ang) + beta[1]], 1)
