"""Seeded synthetic inputs shaped like the HERA-like workloads of arXiv:2504.07090.

This module only *draws inputs*: array layouts, channel and LST grids, pixel
grid bounds, sky mode coefficients, gain coefficients, noise, prior widths,
tangent vectors and momenta.  It holds none of the forward model's arithmetic
(no basis functions, no coordinate transforms, no fringes, no beam), so the
FP64 oracle and the CUDA path can both consume its outputs without sharing any
of the computation they are checked on.  It imports nothing else from this
package.

Workloads (Sec. 3.1 "Array Model and Mock Observations" for the array and the
drift-scan; the sizes are the configurations this library is benchmarked on):

  cfg0  7-antenna hexagon, 16 ch 150-160 MHz, 20 LSTs over 1 h, 32x96 px,
        32x16 modes/channel, 200 point sources, complex128 throughout
  cfg1  37-antenna hexagon, 64 ch 140-160 MHz, 60 LSTs, 128x192 px,
        128x128 modes/channel
  cfg2  64 independent problems, antennas {7,19,37}, channels {16,32,64},
        modes 512..16384, 20 LSTs
  cfg3  cfg1 sizes (preconditioner build and HVP workload)
  cfg4  127-antenna hexagon, 128 ch 120-180 MHz, 120 LSTs, 256x384 px,
        256x256 modes/channel, 2000 point sources
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

DEG = math.pi / 180.0
HEX_SPACING_M = 14.6           # Sec. 3.1: 14.6 m hexagonal packing
LATITUDE_RAD = -30.72 * DEG    # Sec. 3.1: HERA latitude / stripe declination
RA_CENTRE_RAD = 30.0 * DEG     # centre of the drift scan (arbitrary origin)
LST_SPAN_RAD = 15.0 * DEG      # 1 h of drift scan
RA_MARGIN_RAD = 16.5 * DEG     # stripe extends past the LST span by this much
DEC_HALF_WIDTH_RAD = 10.0 * DEG
BEAM_FWHM_REF_RAD = 10.0 * DEG
BEAM_REF_HZ = 150e6
NU0_HZ = 150e6
K_BOLTZMANN = 1.380649e-23
C_LIGHT = 299792458.0


@dataclass
class Problem:
    """Geometry and sizes of one forward-model instance (host, float64)."""
    name: str
    ant_enu: np.ndarray            # [n_ant, 3] metres, east/north/up
    freq_hz: np.ndarray            # [n_freq]
    lst_rad: np.ndarray            # [n_lst]
    lat_rad: float
    n_ra: int
    n_dec: int
    ra_min: float
    ra_max: float
    dec_min: float
    dec_max: float
    n_mode_ra: int
    n_mode_dec: int
    n_gain: int = 4
    beam_fwhm_ref_rad: float = BEAM_FWHM_REF_RAD   # <= 0 means isotropic beam
    beam_ref_hz: float = BEAM_REF_HZ
    sigma: float = 1.0             # noise std per real component (Jy)
    n_src: int = 200
    seed: int = 20250409
    beam_type: int = 0             # 0 Gaussian, 1 modified Airy (Eq. airy)
    dish_ew_m: float = 0.0         # Airy aperture diameters
    dish_ns_m: float = 0.0
    n_freq_modes: int = 0          # > 0: sky modes compressed onto this many Legendre orders in frequency
    extra: dict = field(default_factory=dict)

    @property
    def n_ant(self) -> int:
        return int(self.ant_enu.shape[0])

    @property
    def n_bl(self) -> int:
        return self.n_ant * (self.n_ant - 1) // 2

    @property
    def n_freq(self) -> int:
        return int(self.freq_hz.shape[0])

    @property
    def n_lst(self) -> int:
        return int(self.lst_rad.shape[0])

    @property
    def n_pix(self) -> int:
        return self.n_ra * self.n_dec

    @property
    def n_modes(self) -> int:
        return self.n_mode_ra * self.n_mode_dec

    @property
    def n_sky_rows(self) -> int:
        """Leading extent of the sky parameters: channels, or Legendre orders when compressed."""
        return self.n_freq_modes if self.n_freq_modes > 0 else self.n_freq

    @property
    def n_sky_params(self) -> int:
        return self.n_sky_rows * self.n_modes

    @property
    def n_gain_params(self) -> int:
        return 2 * self.n_ant * self.n_gain

    @property
    def n_params(self) -> int:
        return self.n_sky_params + self.n_gain_params

    @property
    def n_vis(self) -> int:
        return self.n_freq * self.n_lst * self.n_bl

    def terms_per_forward(self) -> int:
        """Vis-pixel terms of the discretised RIME (baseline, channel, LST, pixel)."""
        return self.n_bl * self.n_freq * self.n_lst * self.n_pix


def hex_array(side: int, spacing: float = HEX_SPACING_M) -> np.ndarray:
    """Antennas on a flat hexagonal lattice of the given side (7, 19, 37, 127 for 2, 3, 4, 7)."""
    pts = []
    r = side - 1
    for b in range(-r, r + 1):
        for a in range(-r, r + 1):
            if abs(a) <= r and abs(b) <= r and abs(a + b) <= r:
                pts.append((spacing * (a + 0.5 * b), spacing * (math.sqrt(3.0) / 2.0) * b, 0.0))
    arr = np.array(pts, dtype=np.float64)
    order = np.lexsort((arr[:, 0], arr[:, 1]))
    return np.ascontiguousarray(arr[order])


def drift_scan_problem(name: str, hex_side: int, n_freq: int, f_lo: float, f_hi: float,
                       n_lst: int, n_dec: int, n_ra: int, n_mode_ra: int, n_mode_dec: int,
                       n_src: int = 200, seed: int = 20250409, n_gain: int = 4,
                       ant_enu: np.ndarray | None = None) -> Problem:
    """A drift scan through the stripe at the array latitude (Sec. 3.1), 1 h of LST."""
    freqs = np.linspace(f_lo, f_hi, n_freq) if n_freq > 1 else np.array([0.5 * (f_lo + f_hi)])
    cadence = LST_SPAN_RAD / n_lst
    lsts = RA_CENTRE_RAD + (np.arange(n_lst) - 0.5 * (n_lst - 1)) * cadence
    half_ra = 0.5 * LST_SPAN_RAD + RA_MARGIN_RAD
    return Problem(
        name=name,
        ant_enu=hex_array(hex_side) if ant_enu is None else np.ascontiguousarray(ant_enu, dtype=np.float64),
        freq_hz=np.ascontiguousarray(freqs, dtype=np.float64),
        lst_rad=np.ascontiguousarray(lsts, dtype=np.float64),
        lat_rad=LATITUDE_RAD,
        n_ra=n_ra, n_dec=n_dec,
        ra_min=RA_CENTRE_RAD - half_ra, ra_max=RA_CENTRE_RAD + half_ra,
        dec_min=LATITUDE_RAD - DEC_HALF_WIDTH_RAD, dec_max=LATITUDE_RAD + DEC_HALF_WIDTH_RAD,
        n_mode_ra=n_mode_ra, n_mode_dec=n_mode_dec, n_gain=n_gain,
        n_src=n_src, seed=seed)


def config(name: str) -> Problem:
    """The named workloads.  cfg3 shares cfg1's sizes."""
    if name == "cfg0":
        return drift_scan_problem("cfg0", 2, 16, 150e6, 160e6, 20, 32, 96, 32, 16, 200, 20250409)
    if name in ("cfg1", "cfg3"):
        return drift_scan_problem(name, 4, 64, 140e6, 160e6, 60, 128, 192, 128, 128, 200,
                                  20250410 if name == "cfg1" else 20250412)
    if name == "cfg4":
        return drift_scan_problem("cfg4", 7, 128, 120e6, 180e6, 120, 256, 384, 256, 256, 2000, 20250413)
    if name == "tiny":
        # 3 antennas, odd pixel counts that divide no tile size, few channels
        return drift_scan_problem("tiny", 2, 3, 150e6, 156e6, 4, 5, 17, 4, 3, 20, 7,
                                  ant_enu=hex_array(2)[:3])
    if name == "small":
        # several tiles and a ragged tail in every dimension, still seconds on the oracle
        return drift_scan_problem("small", 2, 6, 150e6, 160e6, 5, 21, 46, 16, 8, 50, 11)
    if name == "mid":
        # 19 antennas (tensor-core tile padding), ragged pixel tail
        return drift_scan_problem("mid", 3, 4, 145e6, 155e6, 3, 24, 70, 16, 16, 50, 13)
    if name == "ant37":
        # the cfg1 array (37 antennas: two 64-wide K atoms in the adjoint tiles) on a small
        # grid, 8 equally spaced channels (frequency-recurrence groups), ragged pixel tail
        return drift_scan_problem("ant37", 4, 8, 146e6, 153e6, 3, 20, 58, 16, 8, 50, 17)
    if name == "ha7":
        # drift-scan grid with the LST step equal to 2 RA pixels (5 LSTs 3 deg apart,
        # 32 RA cells of 1.5 deg): the hour-angle form with stride 2; 7-antenna hexagon
        # (21 baselines in 9 distinct vectors), odd declination count
        return drift_scan_problem("ha7", 2, 4, 150e6, 156e6, 5, 9, 32, 8, 4, 20, 21)
    if name == "ha37":
        # the cfg1 array (666 baselines, 63 distinct vectors) with the LST step equal to
        # one RA pixel (10 LSTs, 32 RA cells of 1.5 deg)
        return drift_scan_problem("ha37", 4, 3, 148e6, 152e6, 10, 7, 32, 8, 4, 20, 23)
    if name == "ha37m":
        # ha37 with 16 x 4 = 64 modes per channel (one 64-block of the mass matrix per
        # channel): the hour-angle leapfrog case
        return drift_scan_problem("ha37m", 4, 3, 148e6, 152e6, 10, 7, 32, 16, 4, 20, 23)
    if name == "hafrac2":
        # LST step of 2.5 RA pixels (5 LSTs 3 deg apart, 40 RA cells of 1.2 deg): hour-angle
        # cells of half a pixel, 5 cells per LST step; 7-antenna hexagon
        return drift_scan_problem("hafrac2", 2, 4, 150e6, 156e6, 5, 9, 40, 8, 4, 20, 31)
    if name == "hafrac4":
        # LST step of 0.75 RA pixel (20 LSTs 0.75 deg apart, 48 RA cells of 1 deg, as in the
        # uneven-problem batch): cells of a quarter pixel, 3 per LST step; 19-antenna hexagon
        return drift_scan_problem("hafrac4", 3, 3, 150e6, 155e6, 20, 6, 48, 8, 4, 20, 37)
    if name == "hachunk":
        # 91-antenna hexagon (more antennas than the phasor table's 64 entries; its covering
        # subset fits), 70 LSTs (two passes of at most 64), LST step of half an RA pixel
        return drift_scan_problem("hachunk", 6, 2, 150e6, 153e6, 70, 4, 112, 16, 4, 20, 41)
    if name == "harand":
        # 12 antennas at seeded random east/north/up offsets (66 distinct baselines: two
        # forward M-tiles, the second ragged), LST step equal to one RA pixel
        rng = np.random.default_rng(29)
        ant = np.column_stack([rng.uniform(-40.0, 40.0, 12), rng.uniform(-40.0, 40.0, 12),
                               rng.uniform(-0.5, 0.5, 12)])
        return drift_scan_problem("harand", 2, 3, 150e6, 155e6, 5, 6, 16, 8, 4, 20, 29, ant_enu=ant)
    raise KeyError(name)


BATCH_MODE_SHAPES = [(32, 16), (32, 32), (64, 32), (64, 64), (128, 64), (128, 128)]


def batch_problems(n: int = 64, seed: int = 20250411) -> list[Problem]:
    """cfg2: independent problems of uneven size drawn from a seed."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.choice([2, 3, 4]))            # 7, 19, 37 antennas
        n_freq = int(rng.choice([16, 32, 64]))
        mra, mdec = BATCH_MODE_SHAPES[int(rng.integers(len(BATCH_MODE_SHAPES)))]
        f_lo = 150e6 if n_freq == 16 else 140e6
        out.append(drift_scan_problem(f"cfg2[{k}]", side, n_freq, f_lo, 160e6, 20,
                                      mdec, (3 * mra) // 2, mra, mdec, 200, seed + 1000 + k))
    return out


# ----------------------------------------------------------------------------- draws

def rayleigh_jeans_jy_per_sr(temp_k: float | np.ndarray, nu_hz: float | np.ndarray):
    """Specific intensity of a brightness temperature (footnote of Sec. 4.3 uses the same law)."""
    return 2.0 * K_BOLTZMANN * np.asarray(nu_hz) ** 2 * np.asarray(temp_k) / C_LIGHT ** 2 * 1e26


def _ra_wavenumber(m: np.ndarray, n_mode_ra: int) -> np.ndarray:
    k = (m + 1) // 2
    k = np.where(m == n_mode_ra - 1, n_mode_ra // 2, k)
    return np.where(m == 0, 0, k)


@dataclass
class Truth:
    theta: np.ndarray      # [n_params] float64: sky modes (freq, m_ra, n_dec) then gains (ant, k, re/im)
    noise: np.ndarray      # [n_freq, n_lst, n_bl, 2] float64, unit normal per real component


def draw_truth(prob: Problem, seed: int | None = None) -> Truth:
    """Truth parameters and a unit noise realisation.

    Sky, drawn directly in mode space (no map is fitted, so no basis is evaluated here):
      * diffuse: 200 K at 150 MHz mean (mode (0,0)) plus 30 % fluctuations whose
        coefficient std falls as (1+kappa)^-1.5 (1+n)^-1.5 in RA wavenumber kappa and
        Legendre degree n; amplitude scales as (nu/150 MHz)^-2.5;
      * point sources: n_src fluxes from dN/dS ~ S^-2 on [0.1, 10] Jy with spectral
        indices N(-0.8, 0.2); their sum is white in mode space, represented through the
        third-order expansion of (nu/nu0)^alpha in log(nu/nu0) with the exact moment
        covariance sum_s S_s^2 alpha_s^(q+q');
      * 21 cm signal: flat power 10 mK^2, independent per channel.
    Gains: g_i(nu) = sum_k gamma_ik P_k(nu_hat) with gamma_i0 = 1 + 0.05 CN(0,1),
    gamma_ik = 0.05 CN(0,1) for k >= 1.
    With n_freq_modes > 0 the sky is drawn as Legendre-in-frequency coefficients instead
    (_draw_compressed); the 21 cm part, white across channels, has no place there.
    """
    rng = np.random.default_rng(prob.seed if seed is None else seed)
    F, M, N = prob.n_freq, prob.n_mode_ra, prob.n_mode_dec
    nk = M * N
    m_idx = np.arange(M)[:, None]
    n_idx = np.arange(N)[None, :]
    kappa = _ra_wavenumber(m_idx, M)
    mean_i = rayleigh_jeans_jy_per_sr(200.0, NU0_HZ)
    std_diff = 0.3 * mean_i * (1.0 + kappa) ** -1.5 * (1.0 + n_idx) ** -1.5
    a_diff = std_diff * rng.standard_normal((M, N))
    a_diff[0, 0] = mean_i
    # point sources
    u = rng.random(prob.n_src)
    s_min, s_max = 0.1, 10.0
    flux = 1.0 / (1.0 / s_min - u * (1.0 / s_min - 1.0 / s_max))
    alpha = rng.normal(-0.8, 0.2, prob.n_src)
    stripe_sr = (prob.ra_max - prob.ra_min) * (math.sin(prob.dec_max) - math.sin(prob.dec_min))
    res_sr = stripe_sr / nk
    mom = np.array([[np.sum(flux ** 2 * alpha ** (q + r)) for r in range(4)] for q in range(4)])
    chol = np.linalg.cholesky(mom + 1e-30 * np.eye(4))
    z = rng.standard_normal((4, nk))
    u_q = (chol @ z) / (res_sr * math.sqrt(nk))           # [4, nk]
    theta = np.empty(prob.n_params, dtype=np.float64)
    if prob.n_freq_modes > 0:
        return _draw_compressed(prob, rng, theta, a_diff.reshape(nk), u_q)
    sky = theta[: F * nk].reshape(F, nk)
    for f, nu in enumerate(prob.freq_hz):
        lg = math.log(nu / NU0_HZ)
        ps = u_q[0] + lg * u_q[1] + lg ** 2 / 2.0 * u_q[2] + lg ** 3 / 6.0 * u_q[3]
        sig21 = rayleigh_jeans_jy_per_sr(math.sqrt(10e-6), nu)
        a21 = sig21 * np.sqrt((2.0 * n_idx + 1.0) / nk) * rng.standard_normal((M, N))
        sky[f] = ((nu / NU0_HZ) ** -2.5 * a_diff + a21).reshape(nk) + ps
    return _draw_gains_and_noise(prob, rng, theta)


def _draw_gains_and_noise(prob: Problem, rng, theta: np.ndarray) -> Truth:
    g = theta[prob.n_sky_params:].reshape(prob.n_ant, prob.n_gain, 2)
    g[:] = 0.05 / math.sqrt(2.0) * rng.standard_normal((prob.n_ant, prob.n_gain, 2))
    g[:, 0, 0] += 1.0
    noise = rng.standard_normal((prob.n_freq, prob.n_lst, prob.n_bl, 2))
    return Truth(theta=theta, noise=noise)


def _draw_compressed(prob: Problem, rng, theta: np.ndarray, a_diff: np.ndarray, u_q: np.ndarray) -> Truth:
    """Sky coefficients of the Legendre-in-frequency model, drawn directly (no basis is
    evaluated): order 0 holds the band's mean sky (the diffuse modes and the point sources'
    flux at 150 MHz); order k >= 1 holds an independent draw of the same angular spectra,
    scaled by 0.2^k, so that the spectra are smooth and the higher orders fall off as a
    power law's expansion does over a narrow band."""
    K, nk = prob.n_freq_modes, prob.n_modes
    sky = theta[: K * nk].reshape(K, nk)
    sky[0] = a_diff + u_q[0]
    scale = np.abs(a_diff).copy()
    scale[0] = 0.3 * abs(a_diff[0])
    for k in range(1, K):
        sky[k] = 0.2 ** k * (scale * rng.standard_normal(nk) + u_q[min(k, 3)])
    return _draw_gains_and_noise(prob, rng, theta)


def with_freq_modes(prob: Problem, n_freq_modes: int) -> Problem:
    """The same problem with its sky compressed onto n_freq_modes Legendre orders in frequency."""
    if not 0 <= n_freq_modes <= prob.n_freq:
        raise ValueError("n_freq_modes must lie in [0, n_freq]")
    return replace(prob, n_freq_modes=int(n_freq_modes), name=f"{prob.name}-K{n_freq_modes}")


def prior_for(prob: Problem, theta_true: np.ndarray, sky_frac: float = 0.05,
              gain_std: float = 0.05) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian prior (mean, inverse variance): 5 % of each channel's rms for sky modes
    (the ~5 % foreground prior of Sec. 3.2), 0.05 for gain coefficients."""
    mu = theta_true.copy()
    lam = np.empty_like(theta_true)
    F, nk = prob.n_sky_rows, prob.n_modes
    sky = theta_true[: F * nk].reshape(F, nk)
    rms = np.sqrt(np.mean(sky ** 2, axis=1))
    lam[: F * nk] = np.repeat(1.0 / (sky_frac * rms) ** 2, nk)
    lam[F * nk:] = 1.0 / gain_std ** 2
    return mu, lam


def random_vectors(n: int, count: int, seed: int) -> np.ndarray:
    """count independent N(0,1) vectors of length n (HVP probes, momenta)."""
    return np.random.default_rng(seed).standard_normal((count, n))


def random_data(prob: Problem, scale: float, seed: int) -> np.ndarray:
    """Arbitrary complex visibilities [freq, lst, bl, 2] for residual-only tests."""
    return scale * np.random.default_rng(seed).standard_normal((prob.n_freq, prob.n_lst, prob.n_bl, 2))


def with_isotropic_beam(prob: Problem) -> Problem:
    return replace(prob, beam_fwhm_ref_rad=0.0)


# modified Airy beam of a 14 m dish squashed along east-west (Eq. airy gives no diameters;
# these are this library's choice)
AIRY_DISH_EW_M, AIRY_DISH_NS_M = 12.0, 14.0


def with_airy_beam(prob: Problem, dish_ew_m: float = AIRY_DISH_EW_M, dish_ns_m: float = AIRY_DISH_NS_M) -> Problem:
    return replace(prob, beam_type=1, dish_ew_m=dish_ew_m, dish_ns_m=dish_ns_m)
