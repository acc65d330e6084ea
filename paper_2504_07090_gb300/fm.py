"""Python binding of libfm (include/fm.h): argument marshalling only.

Every computation runs in the CUDA library; this module checks tensor devices,
dtypes and shapes, passes raw device pointers and the current torch stream, and turns
non-OK statuses into exceptions.  There is no CPU fallback: importing this module
raises when libfm.so has not been built (``paper_2504_07090_gb300.build.build()``).

``ForwardModel`` owns one handle; ``Chi2Potential`` exposes U(theta) with the
hand-written adjoint as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_int64, c_void_p

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfm.so")

FM_OK, FM_ERR_INVALID_ARG, FM_ERR_ALLOC, FM_ERR_CUDA, FM_ERR_NONFINITE, FM_ERR_TIMEOUT, FM_ERR_NOT_SPD, \
    FM_ERR_UNSUPPORTED, FM_ERR_STATE = range(9)
STATUS_NAMES = ["FM_OK", "FM_ERR_INVALID_ARG", "FM_ERR_ALLOC", "FM_ERR_CUDA", "FM_ERR_NONFINITE", "FM_ERR_TIMEOUT",
                "FM_ERR_NOT_SPD", "FM_ERR_UNSUPPORTED", "FM_ERR_STATE"]
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x1": 2, "bf16x3": 3, "fp16x1": 4, "fp16x3": 5}

# every entry point declared in include/fm.h
EXPORTS = ["fm_create", "fm_destroy", "fm_num_params", "fm_num_vis", "fm_set_data", "fm_set_prior", "fm_forward",
           "fm_forward_pixels", "fm_sky_pixels", "fm_chi2_grad", "fm_hvp", "fm_build_precond", "fm_get_precond_blocks",
           "fm_precond_size", "fm_leapfrog", "fm_precond_apply", "fm_set_profiling", "fm_get_profile",
           "fm_contraction_info", "fm_kernel_launches", "fm_sky_pixels_noalloc", "fm_sync_status",
           "fm_last_error", "fm_create_batch", "fm_batch_create", "fm_batch_leapfrog", "fm_batch_kernels",
           "fm_batch_destroy", "fm_diag_bounded_wait", "fm_hmc_chain", "fm_chain_kernels", "fm_draw_normal",
           "fm_draw_accept_uniform", "fm_set_delay_filter", "fm_set_launch_grids", "fm_get_launch_grids"]
CONTRACTION_FORMS = {0: "direct", 1: "antenna", 2: "hour_angle"}


class FmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


class FmConfig(ctypes.Structure):
    _fields_ = [("n_ant", c_int), ("ant_enu_m", POINTER(c_double)),
                ("n_freq", c_int), ("freq_hz", POINTER(c_double)),
                ("n_lst", c_int), ("lst_rad", POINTER(c_double)),
                ("latitude_rad", c_double),
                ("n_ra", c_int), ("n_dec", c_int),
                ("ra_min", c_double), ("ra_max", c_double), ("dec_min", c_double), ("dec_max", c_double),
                ("n_mode_ra", c_int), ("n_mode_dec", c_int), ("n_gain_modes", c_int),
                ("beam_fwhm_ref_rad", c_double), ("beam_ref_hz", c_double), ("sigma_noise", c_double),
                ("precision", c_int), ("beam_type", c_int), ("n_freq_modes", c_int), ("dish_ew_m", c_double),
                ("dish_ns_m", c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfm.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libfm.so not found at {path}; run paper_2504_07090_gb300.build.build() "
                          "(needs nvcc for sm_103a)")
    L = ctypes.CDLL(path)
    vp = c_void_p
    L.fm_create.argtypes = [POINTER(FmConfig), POINTER(vp)]
    L.fm_destroy.argtypes = [vp]
    L.fm_num_params.argtypes = [vp]
    L.fm_num_params.restype = c_int64
    L.fm_num_vis.argtypes = [vp]
    L.fm_num_vis.restype = c_int64
    L.fm_set_data.argtypes = [vp, vp, vp]
    L.fm_set_prior.argtypes = [vp, vp, vp, vp]
    L.fm_forward.argtypes = [vp, vp, vp, vp]
    L.fm_forward_pixels.argtypes = [vp, vp, vp, vp]
    L.fm_sky_pixels.argtypes = [vp, vp, vp, vp]
    L.fm_chi2_grad.argtypes = [vp, vp, vp, vp, vp, vp]
    L.fm_hvp.argtypes = [vp, vp, vp, vp, c_int, vp]
    L.fm_build_precond.argtypes = [vp, vp, c_int, vp]
    L.fm_get_precond_blocks.argtypes = [vp, vp, vp]
    L.fm_precond_size.argtypes = [vp]
    L.fm_precond_size.restype = c_int64
    L.fm_leapfrog.argtypes = [vp, vp, vp, c_double, c_int, c_double, vp, vp, vp]
    L.fm_sync_status.argtypes = [vp, vp]
    L.fm_precond_apply.argtypes = [vp, c_int, vp, vp, vp]
    L.fm_set_profiling.argtypes = [vp, c_int]
    L.fm_get_profile.argtypes = [vp, POINTER(c_double), POINTER(c_int64)]
    L.fm_sky_pixels_noalloc.argtypes = [c_int, c_int, c_int, c_int, c_int, vp, vp, vp, vp, vp]
    L.fm_contraction_info.argtypes = [vp, POINTER(ctypes.c_int32)]
    L.fm_kernel_launches.argtypes = []
    L.fm_kernel_launches.restype = c_int64
    L.fm_last_error.restype = ctypes.c_char_p
    L.fm_create_batch.argtypes = [c_int, POINTER(FmConfig), POINTER(vp)]
    L.fm_batch_create.argtypes = [c_int, POINTER(vp), POINTER(vp), POINTER(vp), POINTER(vp), POINTER(vp), c_int,
                                  POINTER(vp)]
    L.fm_batch_leapfrog.argtypes = [vp, POINTER(c_double), POINTER(c_double), vp]
    L.fm_batch_kernels.argtypes = [vp, POINTER(c_int64)]
    L.fm_batch_destroy.argtypes = [vp]
    L.fm_diag_bounded_wait.argtypes = [c_int64, vp, vp]
    L.fm_hmc_chain.argtypes = [vp, vp, c_int, c_int, c_double, c_double, ctypes.c_uint64, vp, vp, vp]
    L.fm_chain_kernels.argtypes = [vp, POINTER(c_int64)]
    L.fm_set_delay_filter.argtypes = [vp, c_double, c_double]
    L.fm_set_launch_grids.argtypes = [vp, c_int, c_int]
    L.fm_get_launch_grids.argtypes = [vp, POINTER(ctypes.c_int32)]
    L.fm_draw_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, c_int64, vp, c_int, vp]
    L.fm_draw_accept_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, c_int64, vp, vp]
    for name in EXPORTS:
        if name not in ("fm_num_params", "fm_num_vis", "fm_precond_size", "fm_last_error", "fm_kernel_launches"):
            getattr(L, name).restype = c_int
    _lib = L
    return L


def diag_bounded_wait(limit_cycles: int) -> int:
    """Run the bounded-wait diagnostic (fm_diag_bounded_wait); returns the device status."""
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(load().fm_diag_bounded_wait(int(limit_cycles), _ptr(out), _stream()), "fm_diag_bounded_wait")
    return int(out.item())


def draw_normal(seed: int, iteration: int, n: int, dtype=torch.float32) -> torch.Tensor:
    """n standard normals of the chain's momentum draw (fm_draw_normal)."""
    out = torch.empty(n, dtype=dtype, device="cuda")
    _check(load().fm_draw_normal(int(seed), int(iteration), int(n), _ptr(out), 1 if dtype == torch.float64 else 0,
                                 _stream()), "fm_draw_normal")
    return out


def draw_accept_uniform(seed: int, iteration0: int, n: int) -> torch.Tensor:
    """Accept uniforms of iterations iteration0 .. iteration0 + n - 1 (fm_draw_accept_uniform)."""
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(load().fm_draw_accept_uniform(int(seed), int(iteration0), int(n), _ptr(out), _stream()),
           "fm_draw_accept_uniform")
    return out


def kernel_launches() -> int:
    return int(load().fm_kernel_launches())


def last_error() -> str:
    return load().fm_last_error().decode()


def _check(status: int, where: str):
    if status != FM_OK:
        raise FmError(status, where, last_error())


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return c_void_p(0) if t is None else c_void_p(t.data_ptr())


def make_config(prob, precision: str | int = "fp32", sigma: float | None = None):
    """fm_config from a Problem-like object; the returned tuple keeps the host arrays alive."""
    ant = np.ascontiguousarray(prob.ant_enu, dtype=np.float64)
    freq = np.ascontiguousarray(prob.freq_hz, dtype=np.float64)
    lst = np.ascontiguousarray(prob.lst_rad, dtype=np.float64)
    dp = lambda a: a.ctypes.data_as(POINTER(c_double))  # noqa: E731
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg = FmConfig(ant.shape[0], dp(ant), freq.shape[0], dp(freq), lst.shape[0], dp(lst), float(prob.lat_rad),
                   int(prob.n_ra), int(prob.n_dec), float(prob.ra_min), float(prob.ra_max), float(prob.dec_min),
                   float(prob.dec_max), int(prob.n_mode_ra), int(prob.n_mode_dec), int(prob.n_gain),
                   float(prob.beam_fwhm_ref_rad), float(prob.beam_ref_hz),
                   float(prob.sigma if sigma is None else sigma), prec, int(getattr(prob, "beam_type", 0)),
                   int(getattr(prob, "n_freq_modes", 0)), float(getattr(prob, "dish_ew_m", 0.0)),
                   float(getattr(prob, "dish_ns_m", 0.0)))
    return cfg, (ant, freq, lst)


class ForwardModel:
    """One libfm handle bound to the current CUDA device."""

    def __init__(self, prob, precision: str = "fp32", sigma: float | None = None):
        self.lib = load()
        self.precision = precision
        self.prob = prob
        cfg, self._keep = make_config(prob, precision, sigma)
        h = c_void_p()
        _check(self.lib.fm_create(byref(cfg), byref(h)), "fm_create")
        self.h = h
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.n_params = int(self.lib.fm_num_params(h))
        self.n_vis = int(self.lib.fm_num_vis(h))
        self.vis_shape = (prob.n_freq, prob.n_lst, prob.n_bl, 2)
        self.n_sky = (getattr(prob, "n_freq_modes", 0) or prob.n_freq) * prob.n_mode_ra * prob.n_mode_dec
        self.n_pix_total = prob.n_freq * prob.n_ra * prob.n_dec

    def close(self):
        if getattr(self, "h", None):
            self.lib.fm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _t(self, t: torch.Tensor, n: int, name: str):
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"{name}: need a contiguous CUDA {self.dtype} tensor with {n} elements")
        return _ptr(t)

    def empty_vis(self):
        return torch.empty(self.vis_shape, dtype=self.dtype, device="cuda")

    def set_data(self, vis: torch.Tensor):
        _check(self.lib.fm_set_data(self.h, self._t(vis, 2 * self.n_vis, "vis"), _stream()), "fm_set_data")

    def set_prior(self, mu: torch.Tensor, inv_var: torch.Tensor):
        _check(self.lib.fm_set_prior(self.h, self._t(mu, self.n_params, "mu"), self._t(inv_var, self.n_params, "inv_var"),
                                     _stream()), "fm_set_prior")

    def forward(self, theta: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty_vis() if out is None else out
        _check(self.lib.fm_forward(self.h, self._t(theta, self.n_params, "theta"), self._t(out, 2 * self.n_vis, "out"),
                                   _stream()), "fm_forward")
        return out

    def forward_pixels(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty_vis() if out is None else out
        _check(self.lib.fm_forward_pixels(self.h, _ptr(x), self._t(out, 2 * self.n_vis, "out"), _stream()),
               "fm_forward_pixels")
        return out

    def sky_pixels(self, theta: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Pixel maps x[f][dec*n_ra + ra] of the sky modes in theta."""
        out = torch.empty(self.n_pix_total, dtype=self.dtype, device="cuda") if out is None else out
        _check(self.lib.fm_sky_pixels(self.h, self._t(theta, self.n_params, "theta"),
                                      self._t(out, self.n_pix_total, "out"), _stream()), "fm_sky_pixels")
        return out

    def chi2_grad(self, theta: torch.Tensor, grad: torch.Tensor | None = None, scal: torch.Tensor | None = None):
        """Returns (scal, grad): scal = float64 [chi2, U] on the device, grad = grad U."""
        grad = torch.empty(self.n_params, dtype=self.dtype, device="cuda") if grad is None else grad
        scal = torch.empty(2, dtype=torch.float64, device="cuda") if scal is None else scal
        _check(self.lib.fm_chi2_grad(self.h, self._t(theta, self.n_params, "theta"), _ptr(scal),
                                     c_void_p(scal.data_ptr() + 8), self._t(grad, self.n_params, "grad"), _stream()),
               "fm_chi2_grad")
        return scal, grad

    def hvp(self, theta: torch.Tensor, v: torch.Tensor, full: bool = True, out: torch.Tensor | None = None):
        out = torch.empty(self.n_params, dtype=self.dtype, device="cuda") if out is None else out
        _check(self.lib.fm_hvp(self.h, self._t(theta, self.n_params, "theta"), self._t(v, self.n_params, "v"),
                               self._t(out, self.n_params, "out"), 1 if full else 0, _stream()), "fm_hvp")
        return out

    def build_precond(self, theta: torch.Tensor, block: int = 64):
        _check(self.lib.fm_build_precond(self.h, self._t(theta, self.n_params, "theta"), int(block), _stream()),
               "fm_build_precond")

    def precond_blocks(self) -> torch.Tensor:
        n = int(self.lib.fm_precond_size(self.h))
        out = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
        _check(self.lib.fm_get_precond_blocks(self.h, _ptr(out), _stream()), "fm_get_precond_blocks")
        return out[:n]

    def leapfrog(self, q: torch.Tensor, p: torch.Tensor, eps: float, n_steps: int, u: float,
                 h_out: torch.Tensor | None = None, acc_out: torch.Tensor | None = None):
        h_out = torch.empty(2, dtype=torch.float64, device="cuda") if h_out is None else h_out
        acc_out = torch.empty(1, dtype=torch.int32, device="cuda") if acc_out is None else acc_out
        _check(self.lib.fm_leapfrog(self.h, self._t(q, self.n_params, "q"), self._t(p, self.n_params, "p"),
                                    float(eps), int(n_steps), float(u), _ptr(h_out), _ptr(acc_out), _stream()),
               "fm_leapfrog")
        return h_out, acc_out

    def hmc_chain(self, q: torch.Tensor, n_iter: int, n_steps: int, eps0: float, a_min: float, seed: int,
                  state: torch.Tensor, trace: torch.Tensor | None = None) -> torch.Tensor | None:
        """n_iter device-side HMC iterations with the adaptive step (fm_hmc_chain); state is a
        CUDA float64 tensor [2] = (step size, iteration number), updated in place; returns
        trace [n_iter][5] = (eps used, H0, H1, accepted, a) when one is passed."""
        if not (state.is_cuda and state.dtype == torch.float64 and state.numel() == 2 and state.is_contiguous()):
            raise ValueError("state: need a contiguous CUDA float64 tensor of 2 elements")
        if trace is not None and not (trace.is_cuda and trace.dtype == torch.float64 and trace.is_contiguous()
                                      and trace.numel() >= 5 * n_iter):
            raise ValueError("trace: need a contiguous CUDA float64 tensor of at least 5 n_iter elements")
        _check(self.lib.fm_hmc_chain(self.h, self._t(q, self.n_params, "q"), int(n_iter), int(n_steps), float(eps0),
                                     float(a_min), int(seed), _ptr(state), _ptr(trace), _stream()), "fm_hmc_chain")
        return trace

    def set_delay_filter(self, tau_max_s: float = 250e-9, noise_ratio: float = 1e-8):
        """High-pass delay filter of the likelihood (fm_set_delay_filter); tau_max_s <= 0: off."""
        _check(self.lib.fm_set_delay_filter(self.h, float(tau_max_s), float(noise_ratio)), "fm_set_delay_filter")

    def set_launch_grids(self, ctas_fwd: int, ctas_adj: int):
        """CTAs of the hour-angle forward / adjoint contraction kernels (0: one per SM)."""
        _check(self.lib.fm_set_launch_grids(self.h, int(ctas_fwd), int(ctas_adj)), "fm_set_launch_grids")

    def launch_grids(self) -> tuple[int, int]:
        out = (ctypes.c_int32 * 2)()
        _check(self.lib.fm_get_launch_grids(self.h, out), "fm_get_launch_grids")
        return int(out[0]), int(out[1])

    def chain_kernels(self) -> int:
        """Kernel launches one iteration of the captured chain makes (fm_chain_kernels)."""
        out = c_int64()
        _check(self.lib.fm_chain_kernels(self.h, byref(out)), "fm_chain_kernels")
        return int(out.value)

    def precond_apply(self, op: int, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """op 0: L x, 1: L^-1 x, 2: L^-T x, 3: M^-1 x."""
        out = torch.empty_like(x) if out is None else out
        _check(self.lib.fm_precond_apply(self.h, int(op), self._t(x, self.n_params, "in"),
                                         self._t(out, self.n_params, "out"), _stream()), "fm_precond_apply")
        return out

    def set_profiling(self, on: bool = True):
        _check(self.lib.fm_set_profiling(self.h, 1 if on else 0), "fm_set_profiling")

    def get_profile(self):
        """((forward_ms, adjoint_ms), (forward_launches, adjoint_launches)) since the last read."""
        ms = (c_double * 2)()
        cnt = (c_int64 * 2)()
        _check(self.lib.fm_get_profile(self.h, ms, cnt), "fm_get_profile")
        return (ms[0], ms[1]), (int(cnt[0]), int(cnt[1]))

    def contraction_info(self) -> dict:
        """Form of the fringe contraction this handle runs (fm_contraction_info)."""
        out = (ctypes.c_int32 * 4)()
        _check(self.lib.fm_contraction_info(self.h, out), "fm_contraction_info")
        return {"form": CONTRACTION_FORMS[int(out[0])], "fringes": int(out[1]), "lst_step_cells": int(out[2]),
                "hour_angle_cells": int(out[3])}

    def sync_status(self):
        _check(self.lib.fm_sync_status(self.h, _stream()), "fm_sync_status")


class _Chi2Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model):
        scal, grad = model.chi2_grad(theta.detach().contiguous())
        ctx.save_for_backward(grad)
        return scal[1].to(theta.dtype)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return gout * grad, None


def chi2_potential(theta: torch.Tensor, model: ForwardModel) -> torch.Tensor:
    """U(theta) = chi^2/2 + prior as a differentiable scalar; backward uses the CUDA adjoint."""
    return _Chi2Fn.apply(theta, model)


class Batch:
    """One leapfrog trajectory per ForwardModel over independent problems, captured once as a
    single CUDA graph (fm_batch_create) and replayed by run() (fm_batch_leapfrog).  Each chain
    works in place on its own q and p tensors, exactly as ForwardModel.leapfrog does."""

    def __init__(self, models, qs, ps, n_steps: int):
        self.lib = load()
        self.models = list(models)
        n = len(self.models)
        self.n = n
        self.qs, self.ps = list(qs), list(ps)
        self.h_out = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in range(n)]
        self.acc_out = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in range(n)]
        arr = c_void_p * n
        hs = arr(*[m.h for m in self.models])
        qp = arr(*[m._t(q, m.n_params, "q") for m, q in zip(self.models, self.qs)])
        pp = arr(*[m._t(p, m.n_params, "p") for m, p in zip(self.models, self.ps)])
        hp = arr(*[_ptr(t) for t in self.h_out])
        ap = arr(*[_ptr(t) for t in self.acc_out])
        b = c_void_p()
        _check(self.lib.fm_batch_create(n, hs, qp, pp, hp, ap, int(n_steps), byref(b)), "fm_batch_create")
        self.b = b

    def run(self, eps, u):
        """One trajectory per chain with steps eps[k] and accept uniforms u[k]."""
        e = (c_double * self.n)(*[float(x) for x in eps])
        v = (c_double * self.n)(*[float(x) for x in u])
        _check(self.lib.fm_batch_leapfrog(self.b, e, v, _stream()), "fm_batch_leapfrog")
        return self.h_out, self.acc_out

    def kernels(self) -> int:
        out = c_int64()
        _check(self.lib.fm_batch_kernels(self.b, byref(out)), "fm_batch_kernels")
        return int(out.value)

    def close(self):
        if getattr(self, "b", None):
            self.lib.fm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
