"""ctypes loader of the in-tree libglad.so (argument marshalling only).

The library must have been built (``python -m paper_2504_01302_b300.build`` or
``__graft_entry__.build()``); there is no fallback: loading without the shared
object raises."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglad.so")

_p = C.c_void_p
_f = C.POINTER(C.c_float)
_d = C.POINTER(C.c_double)
_i = C.POINTER(C.c_int)
_u8 = C.POINTER(C.c_uint8)


class SystemDesc(C.Structure):
    """Mirror of glad_system_desc in include/glad.h (same field order)."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("ss", C.c_int), ("pix", C.c_double),
        ("data", _f), ("sigma", _f), ("mask", _u8), ("psf_k", C.c_int), ("psf", _f),
        ("src_q", C.c_double), ("src_phi", C.c_double), ("ll_n", C.c_double), ("ll_q", C.c_double),
        ("n_ll2", C.c_int), ("ll2", _d), ("n_sis", C.c_int), ("sis", _d), ("r_soft", C.c_double),
        ("kx", C.c_int), ("ky", C.c_int), ("kss", C.c_int), ("kpix", C.c_double),
        ("kpsf_k", C.c_int), ("kpsf", _f), ("bins", _i), ("n_bins", C.c_int),
        ("v_obs", _f), ("v_sig", _f), ("n_mge_mass", C.c_int), ("n_mge_light", _i),
        ("mge_P", C.c_int), ("n_gl", C.c_int),
        ("mass_rmin", C.c_double), ("mass_rmax", C.c_double),
        ("light_rmin", C.c_double), ("light_rmax", C.c_double),
        ("has_bh", C.c_int), ("bh_sigma", C.c_double), ("L_scale", C.c_double),
        ("n_img", C.c_int), ("img_xy", _d), ("dt_obs", _d), ("dt_sig", _d), ("img_sig", _d),
        ("z_d", C.c_double), ("z_s", C.c_double), ("omega_m", C.c_double), ("kappa_ext", C.c_double),
        ("jam_align", C.c_int), ("sph_nr", C.c_int), ("sph_nw", C.c_int), ("sph_nlos", C.c_int),
        ("sheet", C.c_int), ("sheet_rc", C.c_double), ("sheet_rt", C.c_double),
        ("sheet_n", C.c_int), ("sheet_rmin", C.c_double), ("sheet_rmax", C.c_double),
        ("distance_mode", C.c_int), ("mass_class", C.c_int), ("ll_wc", C.c_double),
        ("src_pix", C.c_int), ("spx_nx", C.c_int), ("spx_ny", C.c_int),
        ("spx_x0", C.c_double), ("spx_x1", C.c_double), ("spx_y0", C.c_double), ("spx_y1", C.c_double),
        ("spx_lam_lo", C.c_double), ("spx_lam_hi", C.c_double), ("spx_iters", C.c_int),
    ]


# entry points declared in include/glad.h: name -> (restype, argtypes)
SIGNATURES = {
    "glad_create": (C.c_int, [C.POINTER(SystemDesc), C.c_int, C.POINTER(_p)]),
    "glad_destroy": (None, [_p]),
    "glad_loglike": (C.c_int, [_p, _p, _p, C.c_int, _p, _p, _p, _p]),
    "glad_loglike_grad": (C.c_int, [_p, _p, _p, C.c_int, _p, _p, _p, _p, _p]),
    "glad_loglike_static": (C.c_int, [_p, _p, _p, C.c_int, _p, _p, _p, _p]),
    "glad_model_image": (C.c_int, [_p, C.c_int, _p, _p, _p]),
    "glad_vrms": (C.c_int, [_p, C.c_int, _p, _p, _p]),
    "glad_profile": (C.c_int, [_p, C.c_int]),
    "glad_kernel_times": (C.c_int, [_p, C.c_int, _d, _i]),
    "glad_kernel_name": (C.c_char_p, [C.c_int]),
    "glad_autotune": (C.c_int, [_p, _p, _p, C.c_int, C.c_int, _p]),
    "glad_tuning": (C.c_int, [_p, _i, _i]),
    "glad_set_tuning": (C.c_int, [_p, C.c_int, C.c_int]),
    "glad_set_negligible": (C.c_int, [_p, C.c_int]),
    "glad_set_precision": (C.c_int, [_p, C.c_int]),
    "glad_pixsrc": (C.c_int, [_p, _p, _p, C.c_int, _p, _p, _p, _p]),
    "glad_pix_factorizations": (C.c_ulonglong, [_p]),
    "glad_pix_launches": (C.c_ulonglong, [_p]),
    "glad_set_pix_path": (C.c_int, [_p, C.c_int]),
    "glad_jam_evaluations": (C.c_int, [_p, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]),
    "glad_enfw_cse": (C.c_int, [C.c_int, _d, _d, _d]),
    "glad_last_error": (C.c_char_p, []),
}


def load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libglad.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


class GladError(RuntimeError):
    pass


def check(rc, what):
    if rc != 0:
        msg = lib().glad_last_error().decode()
        raise GladError(f"{what} failed with status {rc}: {msg}")
