"""FP64 oracle of the forward model, chi^2, gradient, Hessian-vector products,
Gauss-Newton preconditioner blocks, Cholesky mass matrix and leapfrog of
arXiv:2504.07090.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may call this package; the CUDA library never does,
and the two share no code.  The per-baseline RIME sum and its adjoint run in the
plain C of ``fm_oracle.c``; this file assembles them with numpy, one (channel, LST)
pair at a time, in the order the paper's definitions give:

  model        m_pq = g_p conj(g_q) V_pq                (gain terms, Sec. 2.1)
  chi^2        sum |m - d|^2 / sigma^2                  (Eq. likelihood, diagonal Sigma)
  U            chi^2/2 + sum lam (theta - mu)^2 / 2     (Eq. posterior, Gaussian prior)
  gradient     chain rule of U, written out per baseline (reverse-mode AD, Sec. 2.3)
  HVP          directional derivative of that gradient (full) or J^T J v (Gauss-Newton)
  mass matrix  GN Hessian blocks, Cholesky with prior inflation (App. B)
  leapfrog     kick-drift-kick with M^-1 = L^-T L^-1, K = z^T z / 2, L z = p (App. B)
"""
from __future__ import annotations

import ctypes
import math
from ctypes import POINTER, c_double, c_int, c_void_p

import numpy as np

from .build import build_oracle

_LIB = None


class _Problem(ctypes.Structure):
    _fields_ = [("n_ant", c_int), ("n_freq", c_int), ("n_lst", c_int),
                ("n_ra", c_int), ("n_dec", c_int), ("n_mode_ra", c_int), ("n_mode_dec", c_int),
                ("n_gain", c_int),
                ("ant_enu", POINTER(c_double)), ("freq_hz", POINTER(c_double)), ("lst_rad", POINTER(c_double)),
                ("lat_rad", c_double), ("ra_min", c_double), ("ra_max", c_double),
                ("dec_min", c_double), ("dec_max", c_double),
                ("beam_fwhm_ref_rad", c_double), ("beam_ref_hz", c_double),
                ("beam_type", c_int), ("dish_ew", c_double), ("dish_ns", c_double)]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(build_oracle())
        L.orc_create.restype = c_void_p
        L.orc_create.argtypes = [POINTER(_Problem)]
        L.orc_destroy.argtypes = [c_void_p]
        L.orc_get_geometry.argtypes = [c_void_p] + [POINTER(c_double)] * 7
        L.orc_beam.restype = c_double
        L.orc_beam.argtypes = [c_void_p, c_double, c_double]
        L.orc_beam_dir.restype = c_double
        L.orc_beam_dir.argtypes = [c_void_p, c_double, c_double, c_double, c_double]
        L.orc_bessel_j1.restype = c_double
        L.orc_bessel_j1.argtypes = [c_double]
        L.orc_sky.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double)]
        L.orc_sky_adjoint.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double)]
        L.orc_vis_ft.argtypes = [c_void_p, c_int, c_int, POINTER(c_double), POINTER(c_double)]
        L.orc_vis_one.argtypes = [c_void_p, c_int, c_int, c_int, POINTER(c_double), POINTER(c_double)]
        L.orc_adjoint_ft.argtypes = [c_void_p, c_int, c_int, POINTER(c_double), POINTER(c_double)]
        L.orc_num_threads.restype = c_int
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().orc_num_threads())


def bessel_j1(x: float) -> float:
    """J1 by Bessel's integral (the oracle's own evaluation, for its pins)."""
    return float(lib().orc_bessel_j1(float(x)))


class Oracle:
    """FP64 reference for one problem (any object with the Problem attributes)."""

    def __init__(self, prob):
        L = lib()
        self.prob = prob
        self._ant = np.ascontiguousarray(prob.ant_enu, dtype=np.float64)
        self._freq = np.ascontiguousarray(prob.freq_hz, dtype=np.float64)
        self._lst = np.ascontiguousarray(prob.lst_rad, dtype=np.float64)
        self.A = self._ant.shape[0]
        self.F = self._freq.shape[0]
        self.T = self._lst.shape[0]
        self.R, self.D = int(prob.n_ra), int(prob.n_dec)
        self.M, self.N, self.NG = int(prob.n_mode_ra), int(prob.n_mode_dec), int(prob.n_gain)
        self.npix = self.R * self.D
        self.nk = self.M * self.N
        self.B = self.A * (self.A - 1) // 2
        self.sigma = float(prob.sigma)
        # Legendre-in-frequency compression (Eq. fg_legendre): a(nu_f) = sum_k X_k(nu_f) a~_k
        self.K = int(getattr(prob, "n_freq_modes", 0) or 0)
        self.n_sky_m = self.F * self.nk
        self.n_sky = self.K * self.nk if self.K else self.n_sky_m
        self.n_par = self.n_sky + 2 * self.A * self.NG
        if self.K:
            lo, hi = float(np.min(self._freq)), float(np.max(self._freq))
            nuh = 2.0 * (self._freq - lo) / (hi - lo) - 1.0 if hi > lo else np.zeros(self.F)
            self.Xf = np.polynomial.legendre.legvander(nuh, self.K - 1)     # [F, K]
        self._p = _Problem(self.A, self.F, self.T, self.R, self.D, self.M, self.N, self.NG,
                           _dp(self._ant), _dp(self._freq), _dp(self._lst),
                           float(prob.lat_rad), float(prob.ra_min), float(prob.ra_max),
                           float(prob.dec_min), float(prob.dec_max),
                           float(prob.beam_fwhm_ref_rad), float(prob.beam_ref_hz),
                           int(getattr(prob, "beam_type", 0)), float(getattr(prob, "dish_ew_m", 0.0)),
                           float(getattr(prob, "dish_ns_m", 0.0)))
        self._g = L.orc_create(ctypes.byref(self._p))
        if not self._g:
            raise MemoryError("orc_create failed")
        self.ra_c = np.empty(self.R)
        self.dec_c = np.empty(self.D)
        self.domega = np.empty(self.D)
        self.phi = np.empty((self.R, self.M))
        self.leg = np.empty((self.D, self.N))
        self.s = np.empty((self.T, self.npix, 3))
        self.gleg = np.empty((self.F, max(self.NG, 1)))
        L.orc_get_geometry(self._g, _dp(self.ra_c), _dp(self.dec_c), _dp(self.domega), _dp(self.phi),
                           _dp(self.leg), _dp(self.s), _dp(self.gleg))
        self.gleg = self.gleg[:, : self.NG]
        ij = [(i, j) for i in range(self.A) for j in range(i + 1, self.A)]
        self.bl_i = np.array([p[0] for p in ij], dtype=np.int64)
        self.bl_j = np.array([p[1] for p in ij], dtype=np.int64)

    def __del__(self):
        try:
            if getattr(self, "_g", None):
                lib().orc_destroy(self._g)
                self._g = None
        except Exception:
            pass

    # ------------------------------------------------------------------ pieces
    def beam(self, nu: float, s_up: float) -> float:
        return float(lib().orc_beam(self._g, float(nu), float(s_up)))

    def beam_dir(self, nu: float, e: float, n: float, u: float) -> float:
        """Total-power beam at the unit direction (east, north, up): Gaussian or Airy."""
        return float(lib().orc_beam_dir(self._g, float(nu), float(e), float(n), float(u)))

    def split(self, theta: np.ndarray):
        """Per-channel sky modes a[f, j] (expanded from the Legendre coefficients when the sky is
        compressed in frequency) and the gain coefficients."""
        theta = np.asarray(theta, dtype=np.float64)
        if self.K:
            a = self.Xf @ theta[: self.n_sky].reshape(self.K, self.nk)
        else:
            a = theta[: self.n_sky].reshape(self.F, self.nk)
        gam = theta[self.n_sky:].reshape(self.A, self.NG, 2)
        return a, gam

    def sky_to_params(self, g_sky: np.ndarray) -> np.ndarray:
        """A per-channel sky gradient [F, nk] in the parameters' coordinates (the transpose of
        the expansion when the sky is compressed in frequency), flattened."""
        g_sky = np.asarray(g_sky).reshape(self.F, self.nk)
        return (self.Xf.T @ g_sky).reshape(-1) if self.K else g_sky.reshape(-1)

    def sky_f(self, a_f: np.ndarray) -> np.ndarray:
        a_f = np.ascontiguousarray(a_f, dtype=np.float64)
        x = np.empty(self.npix)
        lib().orc_sky(self._g, _dp(a_f), _dp(x))
        return x

    def sky(self, a: np.ndarray) -> np.ndarray:
        return np.stack([self.sky_f(a[f]) for f in range(a.shape[0])])

    def sky_adjoint_f(self, xbar_f: np.ndarray) -> np.ndarray:
        xbar_f = np.ascontiguousarray(xbar_f, dtype=np.float64)
        out = np.empty(self.nk)
        lib().orc_sky_adjoint(self._g, _dp(xbar_f), _dp(out))
        return out

    def gains(self, gam: np.ndarray) -> np.ndarray:
        """g[f, i] = sum_k (gamma_ik,re + i gamma_ik,im) P_k(nu_hat_f)."""
        gc = gam[..., 0] + 1j * gam[..., 1]          # [A, NG]
        return self.gleg @ gc.T                        # [F, A]

    def vis_ft(self, f: int, t: int, x_f: np.ndarray) -> np.ndarray:
        x_f = np.ascontiguousarray(x_f, dtype=np.float64)
        out = np.empty(2 * self.B)
        lib().orc_vis_ft(self._g, int(f), int(t), _dp(x_f), _dp(out))
        return out[0::2] + 1j * out[1::2]

    def vis_one(self, f: int, t: int, b: int, x_f: np.ndarray) -> complex:
        x_f = np.ascontiguousarray(x_f, dtype=np.float64)
        out = np.empty(2)
        lib().orc_vis_one(self._g, int(f), int(t), int(b), _dp(x_f), _dp(out))
        return complex(out[0], out[1])

    def adjoint_ft(self, f: int, t: int, omega: np.ndarray, xbar_f: np.ndarray) -> None:
        om = np.empty(2 * self.B)
        om[0::2] = omega.real
        om[1::2] = omega.imag
        assert xbar_f.dtype == np.float64 and xbar_f.flags.c_contiguous
        lib().orc_adjoint_ft(self._g, int(f), int(t), _dp(om), _dp(xbar_f))

    def _fts(self, fts):
        if fts is None:
            return [(f, t) for f in range(self.F) for t in range(self.T)]
        return [(int(f), int(t)) for f, t in fts]

    # ------------------------------------------------------------------ model
    def vis(self, x: np.ndarray, fts=None) -> np.ndarray:
        V = np.zeros((self.F, self.T, self.B), dtype=np.complex128)
        for f, t in self._fts(fts):
            V[f, t] = self.vis_ft(f, t, x[f])
        return V

    def model(self, theta: np.ndarray, fts=None) -> np.ndarray:
        a, gam = self.split(theta)
        g = self.gains(gam)
        out = np.zeros((self.F, self.T, self.B), dtype=np.complex128)
        xs = {}
        for f, t in self._fts(fts):
            if f not in xs:
                xs[f] = self.sky_f(a[f])
            V = self.vis_ft(f, t, xs[f])
            out[f, t] = g[f, self.bl_i] * np.conj(g[f, self.bl_j]) * V
        return out

    def prior_terms(self, theta, mu, lam):
        if lam is None:
            return 0.0, np.zeros(self.n_par)
        dv = np.asarray(theta, dtype=np.float64) - (0.0 if mu is None else np.asarray(mu, dtype=np.float64))
        return 0.5 * float(np.sum(lam * dv * dv)), lam * dv

    def grad_from_weights(self, theta, s_w):
        """Gradient of chi^2 / 2 for per-visibility residual weights s_w[f, t, b] (the derivative
        of chi^2 / 2 with respect to the conjugate model visibility): the chain rule through the
        gains and the sky of the RIME sum (Sec. 2.3), as in chi2_grad with s_w = r / sigma^2."""
        a, gam = self.split(theta)
        g = self.gains(gam)
        grad = np.zeros(self.n_par)
        gsky = np.zeros((self.F, self.nk))
        ggain = np.zeros((self.A, self.NG, 2))
        bi, bj = self.bl_i, self.bl_j
        for f in range(self.F):
            x_f = self.sky_f(a[f])
            xbar = np.zeros(self.npix)
            X = self.gleg[f]
            for t in range(self.T):
                V = self.vis_ft(f, t, x_f)
                sw = s_w[f, t]
                self.adjoint_ft(f, t, np.conj(g[f, bi]) * g[f, bj] * sw, xbar)
                ti = np.conj(sw) * np.conj(g[f, bj]) * V
                tj = np.conj(sw) * g[f, bi] * V
                for k in range(self.NG):
                    np.add.at(ggain[:, k, 0], bi, X[k] * ti.real)
                    np.add.at(ggain[:, k, 1], bi, -X[k] * ti.imag)
                    np.add.at(ggain[:, k, 0], bj, X[k] * tj.real)
                    np.add.at(ggain[:, k, 1], bj, X[k] * tj.imag)
            gsky[f] += self.sky_adjoint_f(xbar)
        grad[: self.n_sky] = self.sky_to_params(gsky)
        grad[self.n_sky:] += ggain.reshape(-1)
        return grad

    def chi2_grad_filtered(self, theta, d, Fm, mu=None, lam=None):
        """chi^2, U and grad U with the delay filter applied along frequency to the model and the
        data (Eq. rime_filter): r~ = F (m - d) for every (LST, baseline), chi^2 = sum |r~|^2 / N~_ff
        with the diagonal of the filtered noise N~ = F N F^T, N = sigma^2 I (Eq. filtered_noise),
        and the gradient through the residual weights F^T (r~ / N~)."""
        r = self.model(theta) - d
        rt = np.einsum("fg,gtb->ftb", Fm, r)
        ntil = self.sigma ** 2 * np.sum(Fm * Fm, axis=1)
        chi2 = float(np.sum((rt.real ** 2 + rt.imag ** 2) / ntil[:, None, None]))
        s_w = np.einsum("gf,gtb->ftb", Fm, rt / ntil[:, None, None])
        grad = self.grad_from_weights(theta, s_w)
        U = 0.5 * chi2
        pu, pg = self.prior_terms(theta, mu, lam)
        return chi2, U + pu, grad + pg

    def chi2_grad(self, theta, d, mu=None, lam=None, fts=None):
        """chi^2, U = chi^2/2 + prior, and grad U.  With ``fts`` only those (channel, LST)
        pairs contribute (the prior is then left out)."""
        a, gam = self.split(theta)
        g = self.gains(gam)
        grad = np.zeros(self.n_par)
        gsky = np.zeros((self.F, self.nk))
        ggain = np.zeros((self.A, self.NG, 2))
        chi2 = 0.0
        s2 = self.sigma ** 2
        bi, bj = self.bl_i, self.bl_j
        by_f = {}
        for f, t in self._fts(fts):
            by_f.setdefault(f, []).append(t)
        for f, ts in by_f.items():
            x_f = self.sky_f(a[f])
            xbar = np.zeros(self.npix)
            X = self.gleg[f]
            for t in ts:
                V = self.vis_ft(f, t, x_f)
                m = g[f, bi] * np.conj(g[f, bj]) * V
                r = m - d[f, t]
                chi2 += float(np.sum(r.real ** 2 + r.imag ** 2)) / s2
                omega = np.conj(g[f, bi]) * g[f, bj] * r / s2
                self.adjoint_ft(f, t, omega, xbar)
                ti = np.conj(r) * np.conj(g[f, bj]) * V / s2
                tj = np.conj(r) * g[f, bi] * V / s2
                for k in range(self.NG):
                    np.add.at(ggain[:, k, 0], bi, X[k] * ti.real)
                    np.add.at(ggain[:, k, 1], bi, -X[k] * ti.imag)
                    np.add.at(ggain[:, k, 0], bj, X[k] * tj.real)
                    np.add.at(ggain[:, k, 1], bj, X[k] * tj.imag)
            gsky[f] += self.sky_adjoint_f(xbar)
        grad[: self.n_sky] = self.sky_to_params(gsky)
        grad[self.n_sky:] += ggain.reshape(-1)
        U = 0.5 * chi2
        if fts is None:
            pu, pg = self.prior_terms(theta, mu, lam)
            U += pu
            grad += pg
        return chi2, U, grad

    def hvp(self, theta, d, v, lam=None, full: bool = True, fts=None):
        """H v for U: full Hessian (directional derivative of grad U) or Gauss-Newton."""
        a, gam = self.split(theta)
        va, vgam = self.split(v)
        g = self.gains(gam)
        dg = self.gains(vgam)
        out = np.zeros(self.n_par)
        osky = np.zeros((self.F, self.nk))
        ggain = np.zeros((self.A, self.NG, 2))
        s2 = self.sigma ** 2
        bi, bj = self.bl_i, self.bl_j
        by_f = {}
        for f, t in self._fts(fts):
            by_f.setdefault(f, []).append(t)
        for f, ts in by_f.items():
            x_f = self.sky_f(a[f])
            xv_f = self.sky_f(va[f])
            xbar = np.zeros(self.npix)
            X = self.gleg[f]
            gi, gj, dgi, dgj = g[f, bi], g[f, bj], dg[f, bi], dg[f, bj]
            for t in ts:
                V = self.vis_ft(f, t, x_f)
                dV = self.vis_ft(f, t, xv_f)
                r = gi * np.conj(gj) * V - d[f, t]
                dm = dgi * np.conj(gj) * V + gi * np.conj(dgj) * V + gi * np.conj(gj) * dV
                Fb = np.conj(dm) * gi * np.conj(gj)
                ci = np.conj(dm) * np.conj(gj) * V
                cj = np.conj(dm) * gi * V
                if full:
                    Fb = Fb + np.conj(r) * (dgi * np.conj(gj) + gi * np.conj(dgj))
                    ci = ci + np.conj(r) * (np.conj(dgj) * V + np.conj(gj) * dV)
                    cj = cj + np.conj(r) * (dgi * V + gi * dV)
                # Re[F K] = Re[conj(omega) K] with omega = conj(F)
                self.adjoint_ft(f, t, np.conj(Fb) / s2, xbar)
                ci, cj = ci / s2, cj / s2
                for k in range(self.NG):
                    np.add.at(ggain[:, k, 0], bi, X[k] * ci.real)
                    np.add.at(ggain[:, k, 1], bi, -X[k] * ci.imag)
                    np.add.at(ggain[:, k, 0], bj, X[k] * cj.real)
                    np.add.at(ggain[:, k, 1], bj, X[k] * cj.imag)
            osky[f] += self.sky_adjoint_f(xbar)
        out[: self.n_sky] = self.sky_to_params(osky)
        out[self.n_sky:] += ggain.reshape(-1)
        if lam is not None and fts is None:
            out += lam * np.asarray(v, dtype=np.float64)
        return out

    # --------------------------------------------------------------- Jacobian
    def sky_column_response(self, f: int, k: int) -> np.ndarray:
        """dV[t, b] / d a[f, k]: the forward sum with the k-th basis map as the sky."""
        m, n = divmod(k, self.N)
        basis = (self.leg[:, n][:, None] * self.phi[:, m][None, :]).reshape(self.npix)
        return np.stack([self.vis_ft(f, t, basis) for t in range(self.T)])

    def jacobian(self, theta) -> np.ndarray:
        """Full complex Jacobian dm / dtheta, rows (f, t, b), for tiny problems."""
        a, gam = self.split(theta)
        g = self.gains(gam)
        bi, bj = self.bl_i, self.bl_j
        J = np.zeros((self.F, self.T, self.B, self.n_par), dtype=np.complex128)
        for f in range(self.F):
            x_f = self.sky_f(a[f])
            Vf = np.stack([self.vis_ft(f, t, x_f) for t in range(self.T)])     # [T, B]
            gg = g[f, bi] * np.conj(g[f, bj])
            for k in range(self.nk):
                col = gg[None, :] * self.sky_column_response(f, k)
                if self.K:          # the coefficient a~[l, k] enters channel f with weight X_l(nu_f)
                    for l in range(self.K):
                        J[f, :, :, l * self.nk + k] = self.Xf[f, l] * col
                else:
                    J[f, :, :, f * self.nk + k] = col
            X = self.gleg[f]
            for kk in range(self.NG):
                for c, unit in ((0, 1.0), (1, 1j)):
                    for i in range(self.A):
                        col = self.n_sky + (i * self.NG + kk) * 2 + c
                        dgi = np.where(bi == i, X[kk] * unit, 0.0)
                        dgj = np.where(bj == i, X[kk] * unit, 0.0)
                        J[f, :, :, col] = (dgi * np.conj(g[f, bj]) + g[f, bi] * np.conj(dgj))[None, :] * Vf
        return J.reshape(self.F * self.T * self.B, self.n_par)

    def gn_blocks(self, theta, lam=None, bs: int = 64, blocks=None):
        """Gauss-Newton Hessian of U, Re(J^H J)/sigma^2 + diag(lam), on the block-diagonal:
        consecutive sky blocks of size bs inside each channel (inside each Legendre order when
        the sky is compressed in frequency: there the block of order l sums the channels' blocks
        with the weights X_l(nu_f)^2, since channels share no visibility), then the dense gain
        block.  ``blocks`` restricts the sky blocks computed (list of block indices)."""
        a, gam = self.split(theta)
        g = self.gains(gam)
        bi, bj = self.bl_i, self.bl_j
        s2 = self.sigma ** 2
        nb_f = self.nk // bs
        n_lead = self.K if self.K else self.F
        want = range(n_lead * nb_f) if blocks is None else blocks

        memo = {}

        def channel_block(f, j0):
            if (f, j0) not in memo:
                gg = g[f, bi] * np.conj(g[f, bj])
                cols = np.stack([(gg[None, :] * self.sky_column_response(f, j0 * bs + c)).reshape(-1)
                                 for c in range(bs)], axis=1)                  # [T*B, bs]
                memo[(f, j0)] = (cols.conj().T @ cols).real / s2
            return memo[(f, j0)]

        out = {}
        for blk in want:
            l, j0 = divmod(int(blk), nb_f)
            if self.K:
                H = sum(self.Xf[f, l] ** 2 * channel_block(f, j0) for f in range(self.F))
            else:
                H = channel_block(l, j0)
            if lam is not None:
                base = l * self.nk + j0 * bs
                H = H + np.diag(lam[base:base + bs])
            out[int(blk)] = H
        # dense gain block
        ng = 2 * self.A * self.NG
        Hg = np.zeros((ng, ng))
        for f in range(self.F):
            x_f = self.sky_f(a[f])
            X = self.gleg[f]
            for t in range(self.T):
                V = self.vis_ft(f, t, x_f)
                Jg = np.zeros((self.B, ng), dtype=np.complex128)
                for kk in range(self.NG):
                    for c, unit in ((0, 1.0), (1, 1j)):
                        for i in range(self.A):
                            col = (i * self.NG + kk) * 2 + c
                            dgi = np.where(bi == i, X[kk] * unit, 0.0)
                            dgj = np.where(bj == i, X[kk] * unit, 0.0)
                            Jg[:, col] = (dgi * np.conj(g[f, bj]) + g[f, bi] * np.conj(dgj)) * V
                Hg += (Jg.conj().T @ Jg).real / s2
        if lam is not None:
            Hg += np.diag(lam[self.n_sky:])
        return out, Hg


# ------------------------------------------------------------- Eq. gpr
def delay_filter(freq_hz, tau_max_s: float, noise_ratio: float) -> np.ndarray:
    """The Gaussian-process high-pass filter of Eq. gpr, F = I - C_fg (C_fg + C_noise)^-1, with
    C_fg[k, l] = sinc(2 tau_max (nu_k - nu_l)) (a top-hat of half-width tau_max in delay;
    numpy's sinc(x) = sin(pi x) / (pi x)) and C_noise = noise_ratio * C_fg(0) I."""
    nu = np.asarray(freq_hz, dtype=np.float64)
    C = np.sinc(2.0 * tau_max_s * (nu[:, None] - nu[None, :]))
    N = noise_ratio * np.eye(nu.size)
    return np.eye(nu.size) - C @ np.linalg.inv(C + N)


# --------------------------------------------------------------------- App. B
def cholesky_with_inflation(H_lik: np.ndarray, lam_block: np.ndarray, grow: float = 1.1, tries: int = 200):
    """Lower Cholesky factor of H_lik + c diag(lam) for the first c in 1, 1.1, 1.21, ...
    that is positive definite (prior inflation of App. B).  Returns (L, c)."""
    c = 1.0
    for _ in range(tries):
        try:
            return np.linalg.cholesky(H_lik + c * np.diag(lam_block)), c
        except np.linalg.LinAlgError:
            c *= grow
    raise np.linalg.LinAlgError("not SPD after prior inflation")


class BlockCholesky:
    """Mass matrix M = L L^T, block diagonal: list of (start, L_block)."""

    def __init__(self, blocks):
        self.blocks = [(int(s), np.asarray(L, dtype=np.float64)) for s, L in blocks]

    def solve_lower(self, p):            # z = L^-1 p
        import scipy.linalg as sl
        z = np.empty_like(p)
        for s, L in self.blocks:
            z[s:s + L.shape[0]] = sl.solve_triangular(L, p[s:s + L.shape[0]], lower=True)
        return z

    def solve_upper_t(self, z):          # y = L^-T z
        import scipy.linalg as sl
        y = np.empty_like(z)
        for s, L in self.blocks:
            y[s:s + L.shape[0]] = sl.solve_triangular(L.T, z[s:s + L.shape[0]], lower=False)
        return y

    def mul_lower(self, p0):             # p = L p0
        p = np.empty_like(p0)
        for s, L in self.blocks:
            p[s:s + L.shape[0]] = L @ p0[s:s + L.shape[0]]
        return p


def leapfrog(grad_fn, q0, p0, eps: float, n_steps: int, u: float, mass: BlockCholesky):
    """One Hessian-preconditioned HMC trajectory (App. B; leapfrog of Neal 2011).

    grad_fn(q) -> (U, grad U).  p0 is the initial momentum (already L times a unit
    normal).  Kinetic energy K = z^T z / 2 with L z = p; drift dq/dt = L^-T z.
    Accept iff u < exp(H0 - H1).  Returns (q_out, p_end, H0, H1, accepted)."""
    q = np.array(q0, dtype=np.float64, copy=True)
    p = np.array(p0, dtype=np.float64, copy=True)
    U, g = grad_fn(q)
    z = mass.solve_lower(p)
    H0 = U + 0.5 * float(z @ z)
    for _ in range(n_steps):
        p = p - 0.5 * eps * g
        q = q + eps * mass.solve_upper_t(mass.solve_lower(p))
        U, g = grad_fn(q)
        p = p - 0.5 * eps * g
    z = mass.solve_lower(p)
    H1 = U + 0.5 * float(z @ z)
    accepted = bool(u < math.exp(min(0.0, H0 - H1))) if H1 > H0 else bool(u < 1.0)
    return (q if accepted else np.array(q0, dtype=np.float64, copy=True)), p, H0, H1, accepted
