"""Python binding of libglad: a context over one or more systems and the batched
log-likelihood, its gradient (as a torch.autograd.Function), the model image and
the binned v_rms.  PyTorch supplies device memory and the current stream only;
every step of the likelihood runs in the library's CUDA kernels."""
import ctypes as C

import numpy as np
import torch

from . import _lib

NTHETA = 23


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr())


class GladContext:
    """Staged systems (glad_create) and the likelihood calls on them.

    ``systems`` is a list of dicts with the keys of glad_system_desc (see
    include/glad.h); arrays are converted to the expected dtypes."""

    def __init__(self, systems):
        self.lib = _lib.lib()
        self.handle = None
        self._keep = []
        descs = (_lib.SystemDesc * len(systems))()
        for d, s in zip(descs, systems):
            self._fill(d, s)
        h = C.c_void_p()
        _lib.check(self.lib.glad_create(descs, len(systems), C.byref(h)), "glad_create")
        self.handle = h
        self._keep = []
        self.n_bins = [int(s["n_bins"]) for s in systems]
        self.shapes = [(int(s["ny"]), int(s["nx"])) for s in systems]

    def _arr(self, a, dt):
        a = np.ascontiguousarray(np.asarray(a), dtype=dt)
        self._keep.append(a)
        return a

    def _fill(self, d, s):
        f32, f64, i32 = np.float32, np.float64, np.int32
        d.nx, d.ny, d.ss, d.pix = int(s["nx"]), int(s["ny"]), int(s["ss"]), float(s["pix"])
        d.data = _ptr(self._arr(s["data"], f32), C.c_float)
        d.sigma = _ptr(self._arr(s["sigma"], f32), C.c_float)
        d.mask = _ptr(self._arr(s["mask"], np.uint8), C.c_uint8)
        psf = self._arr(s["psf"], f32)
        d.psf_k, d.psf = psf.shape[0], _ptr(psf, C.c_float)
        d.src_q, d.src_phi = float(s["src_q"]), float(s["src_phi"])
        d.ll_n, d.ll_q = float(s["ll_n"]), float(s["ll_q"])
        ll2 = self._arr(np.asarray(s["ll2"]).reshape(-1, 4), f64)
        d.n_ll2, d.ll2 = ll2.shape[0], _ptr(ll2, C.c_double)
        sis = self._arr(np.asarray(s["sis"]).reshape(-1, 3), f64)
        d.n_sis, d.sis = sis.shape[0], _ptr(sis, C.c_double)
        d.r_soft = float(s["r_soft"])
        d.kx, d.ky, d.kss, d.kpix = int(s["kx"]), int(s["ky"]), int(s["kss"]), float(s["kpix"])
        kpsf = self._arr(s["kpsf"], f32)
        d.kpsf_k, d.kpsf = kpsf.shape[0], _ptr(kpsf, C.c_float)
        d.bins = _ptr(self._arr(s["bins"], i32), C.c_int)
        d.n_bins = int(s["n_bins"])
        d.v_obs = _ptr(self._arr(s["v_obs"], f32), C.c_float)
        d.v_sig = _ptr(self._arr(s["v_sig"], f32), C.c_float)
        d.n_mge_mass = int(s["n_mge_mass"])
        d.n_mge_light = _ptr(self._arr(s["n_mge_light"], i32), C.c_int)
        d.mge_P, d.n_gl = int(s["mge_P"]), int(s["n_gl"])
        d.mass_rmin, d.mass_rmax = float(s["mass_rmin"]), float(s["mass_rmax"])
        d.light_rmin, d.light_rmax = float(s["light_rmin"]), float(s["light_rmax"])
        d.has_bh, d.bh_sigma, d.L_scale = int(bool(s["has_bh"])), float(s["bh_sigma"]), float(s["L_scale"])
        img = self._arr(s["img_xy"], f64)
        d.n_img, d.img_xy = img.shape[0], _ptr(img, C.c_double)
        d.dt_obs = _ptr(self._arr(s["dt_obs"], f64), C.c_double)
        d.dt_sig = _ptr(self._arr(s["dt_sig"], f64), C.c_double)
        if s.get("img_sig") is not None:
            d.img_sig = _ptr(self._arr(s["img_sig"], f64), C.c_double)
        d.z_d, d.z_s = float(s["z_d"]), float(s["z_s"])
        d.omega_m, d.kappa_ext = float(s["omega_m"]), float(s["kappa_ext"])
        d.jam_align = int(s.get("jam_align", 0))
        d.sph_nr, d.sph_nw = int(s.get("sph_nr", 0)), int(s.get("sph_nw", 0))
        d.sph_nlos = int(s.get("sph_nlos", 0))
        d.sheet = int(s.get("sheet", 0))
        d.sheet_rc, d.sheet_rt = float(s.get("sheet_rc", 0.0)), float(s.get("sheet_rt", 0.0))
        d.sheet_n = int(s.get("sheet_n", 0))
        d.sheet_rmin, d.sheet_rmax = float(s.get("sheet_rmin", 0.0)), float(s.get("sheet_rmax", 0.0))
        d.distance_mode = int(s.get("distance_mode", 0))
        d.mass_class = int(s.get("mass_class", 0))
        d.ll_wc = float(s.get("ll_wc", 0.0))
        d.src_pix = int(s.get("src_pix", 0))
        if d.src_pix:
            d.spx_nx, d.spx_ny = (int(v) for v in s["spx_n"])
            d.spx_x0, d.spx_x1, d.spx_y0, d.spx_y1 = (float(v) for v in s["spx_box"])
            d.spx_lam_lo, d.spx_lam_hi = (float(v) for v in s.get("spx_lam", (0.0, 0.0)))
            d.spx_iters = int(s.get("spx_iters", 0))

    # ------------------------------------------------------------------ calls
    def _check_theta(self, theta, sys_id):
        assert theta.is_cuda and theta.dtype == torch.float64 and theta.shape[-1] == NTHETA
        theta = theta.contiguous()
        B = theta.shape[0]
        if sys_id is None:
            sys_id = torch.zeros(B, dtype=torch.int32, device=theta.device)
        assert sys_id.dtype == torch.int32 and sys_id.is_cuda and sys_id.shape[0] == B
        return theta, sys_id.contiguous(), B

    def loglike(self, theta, sys_id=None, terms=False):
        """logL [B] (float64), status [B] (int32) and optionally the chi^2 terms [B, 4]
        (pixels, dynamics, delays, image positions)."""
        theta, sys_id, B = self._check_theta(theta, sys_id)
        dev = theta.device
        logL = torch.empty(B, dtype=torch.float64, device=dev)
        status = torch.empty(B, dtype=torch.int32, device=dev)
        tr = torch.empty(B, 4, dtype=torch.float64, device=dev) if terms else None
        rc = self.lib.glad_loglike(self.handle, _dptr(sys_id), _dptr(theta), B, _dptr(logL),
                                   _dptr(status), _dptr(tr) if terms else None, _stream())
        _lib.check(rc, "glad_loglike")
        return (logL, status, tr) if terms else (logL, status)

    def loglike_grad(self, theta, sys_id=None, terms=False):
        """logL [B], d logL/d theta [B, 23], status [B] (and the chi^2 terms)."""
        theta, sys_id, B = self._check_theta(theta, sys_id)
        dev = theta.device
        logL = torch.empty(B, dtype=torch.float64, device=dev)
        grad = torch.empty(B, NTHETA, dtype=torch.float64, device=dev)
        status = torch.empty(B, dtype=torch.int32, device=dev)
        tr = torch.empty(B, 4, dtype=torch.float64, device=dev) if terms else None
        rc = self.lib.glad_loglike_grad(self.handle, _dptr(sys_id), _dptr(theta), B, _dptr(logL),
                                        _dptr(grad), _dptr(status), _dptr(tr) if terms else None,
                                        _stream())
        _lib.check(rc, "glad_loglike_grad")
        return (logL, grad, status, tr) if terms else (logL, grad, status)

    def model_image(self, theta, sys=0):
        theta = theta.reshape(NTHETA).contiguous()
        ny, nx = self.shapes[sys]
        img = torch.empty(ny, nx, dtype=torch.float32, device=theta.device)
        _lib.check(self.lib.glad_model_image(self.handle, sys, _dptr(theta), _dptr(img), _stream()),
                   "glad_model_image")
        return img

    def vrms(self, theta, sys=0):
        theta = theta.reshape(NTHETA).contiguous()
        v = torch.empty(self.n_bins[sys], dtype=torch.float32, device=theta.device)
        _lib.check(self.lib.glad_vrms(self.handle, sys, _dptr(theta), _dptr(v), _stream()), "glad_vrms")
        return v

    def pixsrc(self, theta, sys_id=None, want_s=False):
        """Pixelated-source reconstruction (glad_pixsrc): the regularisation lambda that
        maximises the evidence [B], the log-evidence there [B] and, with want_s, s_MP
        [B, 4624] (row b: the first spx_nx * spx_ny entries)."""
        theta, sys_id, B = self._check_theta(theta, sys_id)
        dev = theta.device
        lam = torch.full((B,), float("nan"), dtype=torch.float64, device=dev)
        lnP = torch.full((B,), float("nan"), dtype=torch.float64, device=dev)
        s = torch.zeros(B, 4624, dtype=torch.float64, device=dev) if want_s else None
        _lib.check(self.lib.glad_pixsrc(self.handle, _dptr(sys_id), _dptr(theta), B, _dptr(lam),
                                        _dptr(lnP), _dptr(s) if want_s else None, _stream()),
                   "glad_pixsrc")
        return (lam, lnP, s) if want_s else (lam, lnP)

    def pix_factorizations(self):
        """Cholesky factorisations of F + lambda C since the last call (glad_pix_factorizations)."""
        torch.cuda.synchronize()
        return int(self.lib.glad_pix_factorizations(self.handle))

    def pix_launches(self):
        """Kernel launches of the pixelated-source stage since the last call (glad_pix_launches)."""
        torch.cuda.synchronize()
        return int(self.lib.glad_pix_launches(self.handle))

    def set_pix_path(self, mode):
        """Form of the pixelated source's evidence evaluations (glad_set_pix_path): 0 by batch
        size, 1 one CTA per sample, 2 multi-launch."""
        _lib.check(self.lib.glad_set_pix_path(self.handle, int(mode)), "glad_set_pix_path")

    def autotune(self, theta, sys_id=None, with_grad=False):
        """Time the JAM launch shapes on this batch and keep the fastest (glad_autotune)."""
        theta, sys_id, B = self._check_theta(theta, sys_id)
        _lib.check(self.lib.glad_autotune(self.handle, _dptr(sys_id), _dptr(theta), B,
                                          1 if with_grad else 0, _stream()), "glad_autotune")
        a, b = C.c_int(), C.c_int()
        self.lib.glad_tuning(self.handle, C.byref(a), C.byref(b))
        return {"jam_pts": a.value, "adj_ept": b.value}

    def set_tuning(self, jam_code, adj_ept):
        """Pin the JAM launch shapes (glad_set_tuning)."""
        _lib.check(self.lib.glad_set_tuning(self.handle, int(jam_code), int(adj_ept)), "glad_set_tuning")

    def set_precision(self, mode):
        """Precision of the forward pass (glad_set_precision): 0 FP32 bulk, 1 FP64 lensing,
        2 FP64 lensing and pair sum."""
        _lib.check(self.lib.glad_set_precision(self.handle, int(mode)), "glad_set_precision")

    def set_negligible(self, mode):
        """Negligible-term skipping of the forward JAM pass (glad_set_negligible)."""
        _lib.check(self.lib.glad_set_negligible(self.handle, int(mode)), "glad_set_negligible")

    def jam_evaluations(self, adjoint=False):
        """Integrand evaluations the JAM pair-sum kernel (or, with adjoint, the table
        adjoint) executed in the last call."""
        n, na = C.c_ulonglong(), C.c_ulonglong()
        _lib.check(self.lib.glad_jam_evaluations(self.handle, C.byref(n), C.byref(na)),
                   "glad_jam_evaluations")
        return na.value if adjoint else n.value

    def kernel_times(self):
        """{kernel name: (ms, launches)} recorded since profiling was enabled."""
        n = self.lib.glad_kernel_times(self.handle, 0, None, None)
        ms = (C.c_double * n)()
        nl = (C.c_int * n)()
        self.lib.glad_kernel_times(self.handle, n, ms, nl)
        return {self.lib.glad_kernel_name(i).decode(): (ms[i], nl[i]) for i in range(n) if nl[i]}

    def profile(self, mode=1):
        """glad_profile: 0 off, 1 event pairs per kernel, 2 the same with the lensing and
        dynamics branches serialised on the caller's stream (isolated kernel times)."""
        self.lib.glad_profile(self.handle, int(mode))

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            self.lib.glad_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GladLogL(torch.autograd.Function):
    """logL(theta) with the library's adjoint gradient in backward."""

    @staticmethod
    def forward(ctx, theta, context, sys_id=None):
        logL, grad, status = context.loglike_grad(theta.detach(), sys_id)
        ctx.save_for_backward(grad)
        return logL

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g[:, None] * grad, None, None
