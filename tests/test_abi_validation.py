"""Error behaviour of the C ABI that needs no GPU: glad_create validates every system
descriptor on the host before it touches the device, and the entry points reject null
contexts and empty batches.  Each invalid descriptor differs from a valid one in a single
field."""
import ctypes as C

import numpy as np
import pytest

from . import systems

GLAD_EINVAL, GLAD_EUNSUPPORTED = 1, 5


def _create(mutate):
    from paper_2504_01302_b300 import _lib
    from paper_2504_01302_b300.glad import GladContext
    s = dict(systems.small_system(7))
    mutate(s)
    with pytest.raises(_lib.GladError) as ei:
        GladContext([s])
    return str(ei.value)


def _set(key, value):
    def m(s):
        s[key] = value
    return m


def _pix(**kw):
    def m(s):
        s.update(src_pix=1, spx_n=(10, 10), spx_box=(-0.5, 0.5, -0.5, 0.5))
        s.update(**kw)
    return m


def _sph(**kw):
    def m(s):
        s.update(jam_align=1, **kw)
    return m


@pytest.mark.parametrize("mutate, status, words", [
    (_set("psf", np.ones((4, 4), np.float32) / 16), GLAD_EINVAL, "psf_k must be odd"),
    (_set("kpsf", np.ones((2, 2), np.float32) / 4), GLAD_EINVAL, "kpsf_k must be odd"),
    (_set("nx", 0), GLAD_EINVAL, "bad image geometry"),
    (_set("kss", 0), GLAD_EINVAL, "bad sky geometry"),
    (_set("n_gl", 1), GLAD_EINVAL, "quadrature order"),
    (_set("mass_rmax", 0.001), GLAD_EINVAL, "bad MGE ranges"),
    (_set("img_xy", np.zeros((1, 2))), GLAD_EINVAL, "need >= 2 images"),
    (_set("z_s", 0.1), GLAD_EINVAL, "bad cosmology"),
    (_set("n_mge_light", [1, 4]), GLAD_EINVAL, "n_mge_light < 2"),
    (_set("psf", np.ones((65, 65), np.float32) / 65 ** 2), GLAD_EUNSUPPORTED, "psf_k >"),
    (_set("n_mge_mass", 200), GLAD_EUNSUPPORTED, "n_mge_mass + sheet Gaussians >"),
    (_set("mge_P", 40), GLAD_EUNSUPPORTED, "mge_P >"),
    (_set("n_mge_light", [100, 40]), GLAD_EUNSUPPORTED, "tracer Gaussians >"),
    (_set("img_xy", np.zeros((9, 2))), GLAD_EUNSUPPORTED, "n_img >"),
    (_set("img_sig", np.array([0.005, 0.0, 0.005, 0.005])), GLAD_EINVAL, "img_sig must be positive"),
    (_set("jam_align", 2), GLAD_EINVAL, "jam_align must be 0 or 1"),
    (_sph(sph_nr=3), GLAD_EINVAL, "sph_nr must be"),
    (_sph(sph_nw=1), GLAD_EINVAL, "sph_nw must be"),
    (_sph(sph_nlos=-1), GLAD_EINVAL, "sph_nlos must be"),
    (_sph(sph_nr=128, sph_nw=64), GLAD_EUNSUPPORTED, "sph_nr * sph_nw >"),
    (_sph(sph_nlos=5000), GLAD_EUNSUPPORTED, "sph_nlos >"),
    (_sph(n_gl=512), GLAD_EUNSUPPORTED, "for the spherically aligned model"),
    (_set("sheet", 3), GLAD_EINVAL, "sheet must be 0, 1 or 2"),
    (_set("distance_mode", 2), GLAD_EINVAL, "distance_mode must be 0 or 1"),
    (lambda s: s.update(sheet=1, sheet_rc=50.0, sheet_rt=45.0), GLAD_EINVAL, "sheet radii"),
    (lambda s: s.update(sheet=1, sheet_n=1), GLAD_EINVAL, "sheet_n must be"),
    (lambda s: s.update(sheet=1, sheet_rmin=10.0, sheet_rmax=1.0), GLAD_EINVAL, "bad sheet MGE range"),
    (lambda s: s.update(sheet=1, sheet_n=120), GLAD_EUNSUPPORTED, "n_mge_mass + sheet Gaussians >"),
    (_pix(src_pix=2), GLAD_EINVAL, "src_pix must be 0 or 1"),
    (_pix(spx_n=(2, 10)), GLAD_EINVAL, "source grid needs >= 3 pixels"),
    (_pix(spx_box=(0.5, -0.5, -0.5, 0.5)), GLAD_EINVAL, "bad source grid extent"),
    (_pix(spx_lam=(1.0, 0.5)), GLAD_EINVAL, "regularisation range"),
    (_pix(spx_iters=500), GLAD_EINVAL, "spx_iters must be"),
    (_pix(mask=np.zeros((48, 48), np.uint8)), GLAD_EINVAL, "non-empty mask"),
    (_pix(spx_n=(70, 70)), GLAD_EUNSUPPORTED, "source grid > 4624"),
])
def test_create_rejects_invalid_descriptors(mutate, status, words):
    msg = _create(mutate)
    assert f"status {status}" in msg and words in msg, msg


def test_create_rejects_bin_indices_beyond_n_bins():
    def m(s):
        b = np.array(s["bins"], np.int32, copy=True)
        b[b >= 0] = s["n_bins"]  # every binned spaxel points past the last bin
        s["bins"] = b
    msg = _create(m)
    assert f"status {GLAD_EINVAL}" in msg and "bin index >= n_bins" in msg, msg


def test_entry_points_reject_null_context_and_empty_batch():
    from paper_2504_01302_b300 import _lib
    lib = _lib.lib()
    p = C.c_void_p(8)  # never dereferenced: the checks come first
    assert lib.glad_loglike(None, p, p, 4, p, p, None, None) == GLAD_EINVAL
    assert lib.glad_loglike_grad(None, p, p, 4, p, p, p, None, None) == GLAD_EINVAL
    assert lib.glad_set_negligible(None, 1) == GLAD_EINVAL
    assert lib.glad_set_tuning(None, 4052, 2) == GLAD_EINVAL
    assert lib.glad_pixsrc(None, p, p, 4, p, p, None, None) == GLAD_EINVAL
    assert lib.glad_pix_factorizations(None) == 0
    assert lib.glad_pix_launches(None) == 0
    assert lib.glad_set_pix_path(None, 1) == GLAD_EINVAL
    assert lib.glad_create(None, 1, C.byref(C.c_void_p())) == GLAD_EINVAL
    assert "glad_create" in lib.glad_last_error().decode()
