"""The library's own fit of the composite class's halo (App. B: the elliptical NFW convergence
as 44 cored steep ellipsoids; glad_enfw_cse, no GPU needed) against the projected NFW shape
k(u) = 2 (1 - F(u)) / (u^2 - 1) written out here from its definition, on the fitted range
u in [1e-4, 1e3], and the fit's structure (non-negative amplitudes, log-spaced cores)."""
import ctypes as C
import math

import numpy as np


def _k(u):
    out = []
    for x in u:
        if abs(x - 1.0) < 1e-6:
            out.append(2.0 / 3.0)
        elif x < 1.0:
            e = math.sqrt(1 - x * x)
            out.append(2 * (1 - math.atanh(e) / e) / (x * x - 1))
        else:
            e = math.sqrt(x * x - 1)
            out.append(2 * (1 - math.atan(e) / e) / (x * x - 1))
    return np.array(out)


def test_library_cse_fit_reproduces_the_nfw_profile():
    from paper_2504_01302_b300 import _lib
    lib = _lib.lib()
    a = (C.c_double * 44)()
    s = (C.c_double * 44)()
    err = C.c_double()
    assert lib.glad_enfw_cse(44, a, s, C.byref(err)) == 44
    a, s = np.array(a), np.array(s)
    assert np.all(a >= 0) and np.sum(a > 0) > 20
    assert np.allclose(np.diff(np.log10(s)), 9.0 / 43, rtol=1e-12) and abs(s[0] - 1e-5) < 1e-20
    u = np.geomspace(1e-4, 1e3, 3001)
    fit = np.sum(a[None, :] * (u[:, None] ** 2 + s[None, :] ** 2) ** -1.5, axis=1)
    rel = np.max(np.abs(fit / _k(u) - 1))
    assert rel < 1e-6 and abs(rel - err.value) < 1e-7, (rel, err.value)
    # a buffer that is too small is refused without writing
    assert lib.glad_enfw_cse(10, a.ctypes.data_as(C.POINTER(C.c_double)),
                             s.ctypes.data_as(C.POINTER(C.c_double)), None) == 44


def test_library_and_oracle_fits_agree():
    """The oracle fits its own decomposition (SciPy's non-negative least squares); the two
    differ as functions by at most the sum of their errors, which bounds the composite class's
    parity term (tests/systems.logl_tol_comp)."""
    from oracle import enfw
    from paper_2504_01302_b300 import _lib
    lib = _lib.lib()
    a = (C.c_double * 44)()
    s = (C.c_double * 44)()
    lib.glad_enfw_cse(44, a, s, None)
    a, s = np.array(a), np.array(s)
    ao, so = enfw.cse_decomposition()
    assert np.allclose(s, so, rtol=1e-12)
    u = np.geomspace(1e-4, 1e3, 3001)
    f1 = np.sum(a[None, :] * (u[:, None] ** 2 + s[None, :] ** 2) ** -1.5, axis=1)
    f2 = np.sum(ao[None, :] * (u[:, None] ** 2 + so[None, :] ** 2) ** -1.5, axis=1)
    assert np.max(np.abs(f1 / f2 - 1)) < 4e-7
