/*
 * fm.h -- C ABI of libfm: the visibility forward model, chi^2 gradient, Hessian-vector
 * products, Gauss-Newton preconditioner and Hessian-preconditioned leapfrog of
 * arXiv:2504.07090 (Kern, "A Differentiable, End-to-End Forward Model for 21 cm
 * Cosmology"), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions (every entry point):
 *  - Pointers named dev_* / documented "device" are caller-owned device memory,
 *    contiguous, and must stay valid until the call's stream work completes.  Host
 *    arrays (fm_config) are copied during fm_create.
 *  - Real arrays are float (4 bytes) unless the handle was created with
 *    FM_PREC_FP64_SIMT, in which case they are double.  Complex arrays interleave
 *    (re, im) in that real type.
 *  - Visibility layout: [n_freq][n_lst][n_bl] complex, baseline b enumerates the
 *    antenna pairs (p, q), p < q, row-major (0,1), (0,2), ..., (1,2), ...
 *  - Parameter vector theta (n_params reals): sky modes a[freq][m_ra][n_dec] first (or, with
 *    n_freq_modes = K > 0, their Legendre-in-frequency coefficients a~[k][m_ra][n_dec]), then
 *    gain coefficients gamma[ant][k][re/im].
 *  - All work is enqueued on `stream` (NULL = legacy default stream) and is
 *    asynchronous; outputs are valid once the stream reaches that point.
 *  - A handle owns its device workspace and is not thread-safe: one host thread
 *    and one stream at a time per handle.
 *  - Errors: every call returns an fm_status; the message of the last failure on
 *    the calling thread is available from fm_last_error().  Invalid arguments are
 *    rejected before any work is enqueued.  Conditions only the device can see
 *    (non-finite energy, a wait that timed out) are written to a device status word
 *    and returned by the next fm_sync_status().
 */
#ifndef FM_H
#define FM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FM_API __attribute__((visibility("default")))
#else
#define FM_API
#endif

typedef struct CUstream_st *fm_stream;   /* identical to cudaStream_t */
typedef struct fm_ctx *fm_handle;

typedef enum {
    FM_OK = 0,
    FM_ERR_INVALID_ARG = 1,   /* null pointer, bad size, unsupported combination */
    FM_ERR_ALLOC = 2,         /* device allocation failed */
    FM_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    FM_ERR_NONFINITE = 4,     /* chi^2 or the Hamiltonian was NaN/Inf (trajectory rejected) */
    FM_ERR_TIMEOUT = 5,       /* a device-side wait exceeded its iteration limit */
    FM_ERR_NOT_SPD = 6,       /* a preconditioner block stayed indefinite after inflation */
    FM_ERR_UNSUPPORTED = 7,   /* shape or precision the library does not support */
    FM_ERR_STATE = 8          /* call order: e.g. leapfrog before data were set */
} fm_status;

typedef enum {
    FM_PREC_FP64_SIMT = 0,    /* complex128 throughout, FP64 CUDA-core contraction */
    FM_PREC_FP32_SIMT = 1,    /* FP32 storage and FP32 CUDA-core contraction */
    FM_PREC_BF16X1 = 2,       /* FP32 storage, tcgen05 BF16 contraction, one product */
    FM_PREC_BF16X3 = 3,       /* FP32 storage, tcgen05 BF16 hi/lo split, three products */
    FM_PREC_FP16X1 = 4,       /* FP32 storage, tcgen05 FP16 contraction (power-of-two scaled), one product */
    FM_PREC_FP16X3 = 5        /* FP32 storage, tcgen05 FP16 hi/lo split (scaled), three products */
} fm_precision;

/* Problem description (Sec. 2.1 discretised RIME; Sec. 3 parameterisation).
 * All arrays are host memory and are copied by fm_create. */
typedef struct {
    int n_ant;                   /* antennas, >= 2 (baselines: all pairs p < q) */
    const double *ant_enu_m;     /* [n_ant][3] east, north, up positions in metres */
    int n_freq;                  /* channels, >= 1 */
    const double *freq_hz;       /* [n_freq] channel frequencies in Hz */
    int n_lst;                   /* local sidereal times, >= 1 */
    const double *lst_rad;       /* [n_lst] in radians */
    double latitude_rad;         /* array latitude */
    int n_ra, n_dec;             /* pixel grid: n_dec rows of n_ra cells, pixel = dec*n_ra + ra */
    double ra_min, ra_max;       /* RA cell edges (radians); cells are uniform */
    double dec_min, dec_max;     /* Dec cell edges (radians); cells are uniform */
    int n_mode_ra;               /* RA functions: 1, cos k a, sin k a (k < M/2), cos(M/2 a) */
    int n_mode_dec;              /* Legendre polynomials P_0 .. P_{N-1} in normalised Dec */
    int n_gain_modes;            /* complex Legendre-in-frequency coefficients per antenna */
    double beam_fwhm_ref_rad;    /* Gaussian beam FWHM at beam_ref_hz (scales as 1/nu) */
    double beam_ref_hz;
    double sigma_noise;          /* noise standard deviation per real component (Jy) */
    int precision;               /* fm_precision */
    int beam_type;               /* FM_BEAM_GAUSSIAN (0, the FWHM above) or FM_BEAM_AIRY (1) */
    int n_freq_modes;            /* 0: independent sky modes per channel; K >= 1 (K <= n_freq): the sky
                                    modes of every channel are sum_{k<K} P_k(nu^) a~_k, Legendre
                                    polynomials of the normalised frequency (Eq. fg_legendre), and the
                                    parameters are a~ [K][n_mode_ra][n_mode_dec] then the gains */
    double dish_ew_m, dish_ns_m; /* FM_BEAM_AIRY: aperture diameters along east-west and north-south
                                    (Eq. airy): power beam (2 J1(x) / x)^2 with
                                    x = (D_ns + sin^2(az) (D_ew - D_ns)) sin(za) pi nu / c,
                                    az the azimuth from north through east */
} fm_config;

enum { FM_BEAM_GAUSSIAN = 0, FM_BEAM_AIRY = 1 };

/* Create a handle: validates the configuration, allocates the device workspace and
 * runs the once-per-handle precompute on the device ("cached mode" of App. C):
 * topocentric pixel directions for every LST, cell solid angles, basis tables and
 * the gain frequency basis.  Synchronous.  On failure *out is NULL. */
FM_API fm_status fm_create(const fm_config *cfg, fm_handle *out);

/* Release the handle and all its device memory.  NULL is accepted. */
FM_API fm_status fm_destroy(fm_handle h);

FM_API int64_t fm_num_params(fm_handle h);     /* K*n_mode_ra*n_mode_dec + 2*n_ant*n_gain_modes, K = n_freq_modes
                                                   (n_freq when that is 0) */
FM_API int64_t fm_num_vis(fm_handle h);        /* n_freq*n_lst*n_bl complex visibilities */

/* Data visibilities d (device, [n_freq][n_lst][n_bl] complex) used by the chi^2 of
 * Eq. likelihood with Sigma = sigma_noise^2 I.  Copied into the handle. */
FM_API fm_status fm_set_data(fm_handle h, const void *dev_vis, fm_stream stream);

/* Gaussian prior of Eq. posterior: U gains sum_k inv_var_k (theta_k - mu_k)^2 / 2.
 * dev_mu, dev_inv_var: device [n_params]; copied.  Without a call the prior is zero. */
FM_API fm_status fm_set_prior(fm_handle h, const void *dev_mu, const void *dev_inv_var, fm_stream stream);

/* Model visibilities m_pq = g_p conj(g_q) V_pq(theta) (Eq. rime_discrete with the gain
 * terms of Sec. 2.1), written to dev_vis_out ([n_freq][n_lst][n_bl] complex). */
FM_API fm_status fm_forward(fm_handle h, const void *dev_theta, void *dev_vis_out, fm_stream stream);

/* Unit-gain visibilities V(nu,t) of pixel values dev_x ([n_freq][n_pix] reals, the sky
 * brightness per pixel in Jy/sr) -- Eq. rime_discrete alone, for tests. */
FM_API fm_status fm_forward_pixels(fm_handle h, const void *dev_x, void *dev_vis_out, fm_stream stream);

/* Sky maps of the parameters: x[f][dec][ra] = sum_{m,n} Phi_m(ra) P_n(dec) a[f][m][n]
 * (the separable mode -> pixel transform of Eq. fg_separable / Eq. eor_model) in Jy/sr,
 * dev_x_out: device [n_freq][n_dec*n_ra] reals.  Uses the handle's workspace. */
FM_API fm_status fm_sky_pixels(fm_handle h, const void *dev_theta, void *dev_x_out, fm_stream stream);

/* chi^2 = sum |m - d|^2 / sigma^2 (Eq. likelihood) and the gradient of
 * U = chi^2/2 + prior (the negative log posterior of Eq. posterior up to a constant).
 * dev_chi2_out, dev_u_out: device double[1] (dev_u_out may be NULL).
 * dev_grad_out: device [n_params]. */
FM_API fm_status fm_chi2_grad(fm_handle h, const void *dev_theta, double *dev_chi2_out, double *dev_u_out,
                       void *dev_grad_out, fm_stream stream);

/* Hessian-vector product of U at theta along v: full = 1 gives the full Hessian
 * (equal to a finite difference of the gradient), full = 0 the Gauss-Newton matrix
 * Re(J^H J)/sigma^2 + prior (the mass matrix of Sec. 4.2 / App. B). */
FM_API fm_status fm_hvp(fm_handle h, const void *dev_theta, const void *dev_v, void *dev_hv_out, int full,
                 fm_stream stream);

/* Build the HMC mass matrix at theta (Sec. 4.2, App. B): the Gauss-Newton Hessian of U
 * on a block diagonal -- `block` consecutive sky modes within a channel (block = 64,
 * or 1 for the diagonal; n_mode_ra*n_mode_dec must be a multiple of it) plus one dense
 * block for all gain coefficients (diagonal when block = 1) -- accumulated in FP64,
 * then Cholesky-factored block by block, inflating the prior part by 1.1x per retry
 * until positive definite.  Returns FM_ERR_NOT_SPD after 200 retries. */
FM_API fm_status fm_build_precond(fm_handle h, const void *dev_theta, int block, fm_stream stream);

/* Copy the preconditioner's FP64 Gauss-Newton blocks (before factorisation) to
 * dev_out: sky blocks [n_sky/block][block][block] then the gain block [ng][ng]
 * (ng = 2*n_ant*n_gain_modes; only its diagonal when block = 1, as [ng]). */
FM_API fm_status fm_get_precond_blocks(fm_handle h, double *dev_out, fm_stream stream);
FM_API int64_t fm_precond_size(fm_handle h);   /* doubles written by fm_get_precond_blocks */

/* One Hessian-preconditioned HMC trajectory (App. B; leapfrog of Neal 2011):
 * H0 = U(q) + z.z/2 with L z = p; n_steps of kick(eps/2) - drift(eps L^-T L^-1 p) -
 * kick(eps/2); H1 likewise; accepted iff u_accept < exp(H0 - H1).
 * dev_q (in: q0; out: final q if accepted, q0 otherwise), dev_p (in: initial momentum,
 * already L times a unit normal; out: final momentum): device [n_params].
 * dev_h_out: device double[2] = {H0, H1}; dev_accepted_out: device int[1].
 * Needs fm_set_data and fm_build_precond first (FM_ERR_STATE otherwise). */
FM_API fm_status fm_leapfrog(fm_handle h, void *dev_q, void *dev_p, double eps, int n_steps, double u_accept,
                      double *dev_h_out, int *dev_accepted_out, fm_stream stream);

/* A Markov chain of Hessian-preconditioned HMC iterations run on the device (App. B: the
 * momentum p = L z with z ~ N(0, 1), one leapfrog trajectory, the Metropolis test, and the
 * adaptive step size of App. B).  Each of the n_iter iterations:
 *   1. draws z (n_params normals) and the accept uniform u from the counter-based generator
 *      Philox4x32-10 (Salmon et al., SC 2011) keyed by `seed`, at the iteration number
 *      it = dev_state[1]: see fm_draw_normal and fm_draw_accept_uniform for the exact draws;
 *   2. p = L z (fm_precond_apply op 0) and one fm_leapfrog trajectory of n_steps with step
 *      eps = dev_state[0] and uniform u, in place on dev_q;
 *   3. with a = min(1, exp(H0 - H1)) (0 when H0 or H1 is not finite): eps <- eps / 1.2 if
 *      a < a_min, else eps <- min(eps0, 1.2 eps) (the paper's threshold is a_min = 0.2);
 *      writes {eps used, H0, H1, accepted (0/1), a} to dev_trace[k][0..4] for the k-th
 *      iteration of this call (dev_trace may be NULL), and advances dev_state[1] by 1.
 * dev_q: device [n_params] (the chain state, updated in place); dev_state: device double[2]
 * {step size > 0, iteration number (a whole number)}, read and updated by the device, so a
 * chain continues across calls; dev_trace: device double[n_iter][5] or NULL.
 * The first call for a given (dev_q, dev_state, n_steps) captures one iteration as a CUDA
 * graph (after one chi^2 + gradient evaluation and a synchronisation of `stream`); every
 * iteration is one launch of that graph on `stream`, and nothing is read back to the host.
 * Needs fm_set_data and fm_build_precond first (FM_ERR_STATE otherwise).  A trajectory with a
 * non-finite energy is rejected and raises FM_ERR_NONFINITE at the next fm_sync_status. */
FM_API fm_status fm_hmc_chain(fm_handle h, void *dev_q, int n_iter, int n_steps, double eps0, double a_min,
                              uint64_t seed, double *dev_state, double *dev_trace, fm_stream stream);
/* kernel launches one iteration of the handle's captured chain makes (0 before the first call) */
FM_API fm_status fm_chain_kernels(fm_handle h, int64_t *out);

/* The chain's draws, for use and for checking: element i of the momentum draw at iteration
 * `iteration` comes from the Philox4x32-10 block of counter (i / 4, iteration mod 2^32,
 * iteration / 2^32, 0) and key (seed mod 2^32, seed / 2^32): its four output words w_j give
 * u_j = (floor(w_j / 256) + 1/2) 2^-24, and elements 4g .. 4g+3 are
 * r0 cos(2 pi u1), r0 sin(2 pi u1), r2 cos(2 pi u3), r2 sin(2 pi u3) with r_j = sqrt(-2 ln u_j)
 * (Box-Muller), computed in FP32 and stored as float (fp64 = 0) or double (fp64 = 1) in
 * dev_out[n].  The accept uniform of iteration it is (w_0 + 1/2) 2^-32 of counter
 * (0, it mod 2^32, it / 2^32, 1); fm_draw_accept_uniform writes those of iterations
 * iteration0 .. iteration0 + n - 1 to dev_out[n] (double). */
FM_API fm_status fm_draw_normal(uint64_t seed, uint64_t iteration, int64_t n, void *dev_out, int fp64,
                                fm_stream stream);
FM_API fm_status fm_draw_accept_uniform(uint64_t seed, uint64_t iteration0, int64_t n, double *dev_out,
                                        fm_stream stream);

/* Batched trajectories over independent problems (one HMC chain per handle; App. B for each
 * chain, the chains independent of one another).
 *
 * fm_create_batch: fm_create for cfgs[0..n-1] into out[0..n-1]; on a failure the handles
 * already created are destroyed, out[] is all NULL and the failing status is returned.
 *
 * fm_batch_create: captures, once, one fm_leapfrog trajectory of n_steps for every handle
 * hs[k] on its own state (dev_q[k], dev_p[k], dev_h_out[k], dev_accepted_out[k]: the same
 * meaning, types and sizes as in fm_leapfrog) as parallel branches of one CUDA graph.  Every
 * handle must have had fm_set_data and fm_build_precond (FM_ERR_STATE otherwise); no handle
 * may appear twice.  Before the capture it runs one chi^2 + gradient evaluation per handle
 * at dev_q[k] (so that every buffer the trajectory needs exists) and synchronises; the call
 * allocates the batch's streams, events, graph and a device array of 2 n doubles.  The
 * handles and the four device buffers of every chain must stay valid, and must not be used
 * by other calls while a batch launch runs, until fm_batch_destroy.
 *
 * fm_batch_leapfrog: one launch of the captured graph on `stream`: chain k runs with step
 * eps[k] > 0 and accept uniform u_accept[k] in [0, 1) (host arrays of n; copied before the
 * call returns), from the q and p its buffers hold, with exactly the arithmetic of
 * fm_leapfrog on that handle.  Stream-ordered and asynchronous like fm_leapfrog.
 *
 * fm_batch_destroy: synchronises the device and frees the batch (not the handles). */
typedef struct fm_batch_s *fm_batch;
FM_API fm_status fm_create_batch(int n, const fm_config *cfgs, fm_handle *out);
FM_API fm_status fm_batch_create(int n, const fm_handle *hs, void *const *dev_q, void *const *dev_p,
                                 double *const *dev_h_out, int *const *dev_accepted_out, int n_steps,
                                 fm_batch *out);
FM_API fm_status fm_batch_leapfrog(fm_batch b, const double *eps, const double *u_accept, fm_stream stream);
/* number of kernel launches one fm_batch_leapfrog call makes (kernel nodes of the graph) */
FM_API fm_status fm_batch_kernels(fm_batch b, int64_t *out);
FM_API fm_status fm_batch_destroy(fm_batch b);

/* High-pass delay filter along frequency on the model and the data (Eq. rime_filter), the
 * Gaussian-process filter of Eq. gpr: F = I - C_fg (C_fg + C_noise)^-1 with
 * C_fg[k][l] = sinc(2 tau_max_s (nu_k - nu_l)) (sinc(x) = sin(pi x) / (pi x): a top-hat of
 * half-width tau_max_s seconds in delay) and C_noise = noise_ratio I (the paper: 250 ns and
 * 1e-8), built on the host in FP64 and applied to every (LST, baseline) column.  With it on,
 * fm_chi2_grad (and every trajectory) uses chi^2 = sum |F (m - d)|^2 / N~_ff with the diagonal
 * N~_ff = sigma^2 sum_g F_fg^2 of the filtered noise F N F^T (Eq. filtered_noise), and its
 * gradient.  fm_forward still returns the unfiltered model; fm_hvp returns
 * FM_ERR_UNSUPPORTED; fm_build_precond builds the unfiltered Gauss-Newton mass matrix (any
 * SPD mass matrix keeps the sampler exact).  tau_max_s <= 0 switches the filter off.
 * Synchronous (host build and upload).  FM_ERR_UNSUPPORTED when the channel count exceeds the
 * filter kernel's shared memory (128 channels in FP32, 64 in FP64). */
FM_API fm_status fm_set_delay_filter(fm_handle h, double tau_max_s, double noise_ratio);

/* Apply the preconditioner's block Cholesky factor L (M = L L^T, App. B) to a device
 * vector [n_params]: op 0: out = L in (momentum draw p = L p0);  op 1: out = L^-1 in
 * (z of the kinetic energy);  op 2: out = L^-T in (Laplace-approximation draw from
 * L^T v = v0);  op 3: out = M^-1 in = L^-T L^-1 in (the drift direction).
 * Needs fm_build_precond first (FM_ERR_STATE otherwise).  in and out may not alias. */
FM_API fm_status fm_precond_apply(fm_handle h, int op, const void *dev_in, void *dev_out, fm_stream stream);

/* Event timing of the two contraction kernels (forward fringe sum, pixel adjoint; the
 * main kernel of each, without its operand preparation) on the stream each call uses: fm_set_profiling(h, 1) starts recording, fm_get_profile
 * synchronises, writes total milliseconds and launch counts per class
 * (out_ms[2], out_count[2]: 0 = forward contraction, 1 = adjoint contraction) and
 * clears the record.  Off by default; recording adds two events per contraction. */
FM_API fm_status fm_set_profiling(fm_handle h, int on);
FM_API fm_status fm_get_profile(fm_handle h, double *out_ms, int64_t *out_count);

/* No-allocation variant of fm_sky_pixels (the paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc at call time, such as code running
 * under an allocator it does not own or inside a region where a new device allocation
 * is not allowed).  It takes no handle: the caller passes the basis tables
 * dev_phi [n_ra][n_mode_ra] (RA functions at the cell centres), dev_leg
 * [n_dec][n_mode_dec] (Legendre polynomials at the cell centres), the modes dev_a
 * [n_freq][n_mode_ra][n_mode_dec] and the output dev_x [n_freq][n_dec][n_ra], all float
 * device memory, and the call computes x[f][d][r] = sum_n leg[d][n] sum_m phi[r][m]
 * a[f][m][n] without allocating anything.  The intermediate sum over m lives in a
 * file-scope device array of 2^21 floats (8 MiB) that every GPU loading the library
 * holds until the process exits; n_freq*n_ra*n_mode_dec above 2^21 is rejected with
 * FM_ERR_INVALID_ARG, and so are n_freq > 65535 and n_ra or n_dec > 65535 * 32 (the
 * launch grid), before anything is launched.  The first call on each device looks up the array's device
 * address with that device current (make that first call before any stream capture).
 * Every call shares the array, which keeps the last call's contents: calls that
 * overlap on the GPU (other streams, or a second call before the first finished on a
 * different stream) race on it. */
FM_API fm_status fm_sky_pixels_noalloc(int n_freq, int n_ra, int n_dec, int n_mode_ra, int n_mode_dec,
                                       const float *dev_phi, const float *dev_leg, const float *dev_a, float *dev_x,
                                       fm_stream stream);

/* Which form of the fringe contraction (Eq. rime_discrete) the handle runs, written to
 * out[4] (host int32):
 *   out[0]  0 = direct per-baseline SIMT sum (FP64 / FP32 precisions),
 *           1 = antenna form on the tensor cores (V = E W E^H per channel and LST),
 *           2 = hour-angle form on the tensor cores (drift scan with the LST step k / q RA
 *               pixels, q <= 4: one phasor table per channel over hour-angle cells of
 *               1 / q pixel, the sky as a Toeplitz operand, baselines with equal vectors up
 *               to sign computed once);
 *   out[1]  distinct fringes computed per channel and LST (form 2: baseline groups;
 *           otherwise the number of baselines);
 *   out[2]  LST step in hour-angle cells, k (form 2), else 0;
 *   out[3]  hour-angle cells per declination row, padded (form 2), else 0.
 * The form is fixed at fm_create; the environment variable FM_HA=0 read there
 * disables form 2 and FM_HA_GROUPS=0 makes it compute every baseline separately. */
FM_API fm_status fm_contraction_info(fm_handle h, int32_t *out);

/* Launch grids of the hour-angle contraction kernels (the knobs of the autotuner,
 * paper_2504_07090_gb300/autotune.py; the paper has no counterpart): ctas_fwd CTAs for the
 * forward contraction (its work units are re-partitioned over them) and ctas_adj for the
 * adjoint, each in [1, number of SMs], or 0 for one CTA per SM (the default).  Fewer CTAs let
 * independent handles (the batched schedule) run side by side on the GPU.  The results change
 * only by the order of the partial sums.  FM_ERR_UNSUPPORTED when the handle does not run the
 * hour-angle form.  fm_get_launch_grids writes the grids in use to out[2] (host int32; 0 when
 * the form is off).  Not to be called while work of the handle is in flight or captured. */
FM_API fm_status fm_set_launch_grids(fm_handle h, int ctas_fwd, int ctas_adj);
FM_API fm_status fm_get_launch_grids(fm_handle h, int32_t *out);

/* Diagnostic of the device-side failure path (no counterpart in the paper): one CTA waits,
 * with the bounded mbarrier wait of the tensor-core kernels and a limit of limit_cycles SM
 * clocks (1 .. the kernels' own limit of 4e9), on a barrier that nothing arrives at, then
 * writes FM_ERR_TIMEOUT (or FM_OK had the wait completed) to dev_status_out (device int[1])
 * and returns; nothing faults or hangs and the context stays usable.  Used by the tests of
 * the failure handling. */
FM_API fm_status fm_diag_bounded_wait(int64_t limit_cycles, int *dev_status_out, fm_stream stream);

/* Kernels launched by this library in this process so far (all handles). */
FM_API int64_t fm_kernel_launches(void);

/* Synchronise the stream and return (then clear) the handle's device status word:
 * FM_ERR_NONFINITE or FM_ERR_TIMEOUT if a kernel raised one, else FM_OK. */
FM_API fm_status fm_sync_status(fm_handle h, fm_stream stream);

/* Message of the last non-OK status returned on this thread ("" if none). */
FM_API const char *fm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FM_H */
