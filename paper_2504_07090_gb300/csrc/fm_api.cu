// C ABI of libfm (include/fm.h): argument checks, handle lifetime, device workspace
// and the stage sequence of each entry point.  Every numerical step runs in the
// kernels of k_*.cu; this file only validates, allocates and enqueues.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <type_traits>

#include "fm_internal.cuh"

namespace fm {

static thread_local char g_err[512] = "";
long long g_launches = 0;

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

fm_status cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? FM_ERR_ALLOC : FM_ERR_CUDA;
}

static fm_status invalid(const char *msg)
{
    set_error("invalid argument: %s", msg);
    return FM_ERR_INVALID_ARG;
}

template <typename T>
static fm_status dalloc(Ctx &c, T **p, size_t count)
{
    void *q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(q);
    *p = (T *)q;
    return FM_OK;
}

static fm_status dalloc_bytes(Ctx &c, void **p, size_t bytes)
{
    char *q = nullptr;
    FM_TRY(dalloc<char>(c, &q, bytes));
    *p = q;
    return FM_OK;
}

static void free_ctx(Ctx *c)
{
    if (!c) return;
    chain_release(*c);
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

static bool finite_arr(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

static fm_status validate(const fm_config *cfg)
{
    if (!cfg) return invalid("cfg is NULL");
    if (cfg->n_ant < 2) return invalid("n_ant must be >= 2");
    if (cfg->n_ant > 256) { set_error("n_ant > 256 is not supported"); return FM_ERR_UNSUPPORTED; }
    if (cfg->n_freq < 1 || cfg->n_lst < 1) return invalid("n_freq and n_lst must be >= 1");
    if (cfg->n_ra < 1 || cfg->n_dec < 1) return invalid("n_ra and n_dec must be >= 1");
    if (cfg->n_mode_ra < 1 || cfg->n_mode_dec < 1) return invalid("mode counts must be >= 1");
    if (cfg->n_gain_modes < 1 || cfg->n_gain_modes > 16) return invalid("n_gain_modes must be in [1, 16]");
    if (!cfg->ant_enu_m || !cfg->freq_hz || !cfg->lst_rad) return invalid("a host array is NULL");
    if (!finite_arr(cfg->ant_enu_m, 3 * (size_t)cfg->n_ant) || !finite_arr(cfg->freq_hz, cfg->n_freq) ||
        !finite_arr(cfg->lst_rad, cfg->n_lst))
        return invalid("non-finite value in a host array");
    for (int f = 0; f < cfg->n_freq; ++f)
        if (!(cfg->freq_hz[f] > 0.0)) return invalid("frequencies must be > 0");
    if (!(cfg->ra_max > cfg->ra_min) || !(cfg->dec_max > cfg->dec_min)) return invalid("empty pixel grid range");
    if (cfg->dec_min < -kPi / 2 - 1e-12 || cfg->dec_max > kPi / 2 + 1e-12) return invalid("declination outside [-pi/2, pi/2]");
    if (!std::isfinite(cfg->latitude_rad) || std::fabs(cfg->latitude_rad) > kPi / 2) return invalid("latitude");
    if (!(cfg->sigma_noise > 0.0) || !std::isfinite(cfg->sigma_noise)) return invalid("sigma_noise must be > 0");
    if (cfg->beam_fwhm_ref_rad > 0.0 && !(cfg->beam_ref_hz > 0.0)) return invalid("beam_ref_hz must be > 0");
    if (cfg->beam_type != FM_BEAM_GAUSSIAN && cfg->beam_type != FM_BEAM_AIRY) return invalid("unknown beam_type");
    if (cfg->beam_type == FM_BEAM_AIRY &&
        (!(cfg->dish_ew_m > 0.0) || !(cfg->dish_ns_m > 0.0) || !std::isfinite(cfg->dish_ew_m) ||
         !std::isfinite(cfg->dish_ns_m)))
        return invalid("the Airy beam needs dish_ew_m and dish_ns_m > 0");
    if (cfg->precision < FM_PREC_FP64_SIMT || cfg->precision > FM_PREC_FP16X3) return invalid("precision");
    if (cfg->n_freq_modes < 0 || cfg->n_freq_modes > cfg->n_freq) return invalid("n_freq_modes must be in [0, n_freq]");
    long long npix = (long long)cfg->n_ra * cfg->n_dec;
    if (npix > (1LL << 30) || (long long)cfg->n_mode_ra * cfg->n_mode_dec > (1LL << 30))
        return invalid("grid too large");
    return FM_OK;
}

static fm_status create_impl(const fm_config *cfg, Ctx *c)
{
    c->cfg = *cfg;
    c->A = cfg->n_ant; c->F = cfg->n_freq; c->T = cfg->n_lst;
    c->R = cfg->n_ra; c->D = cfg->n_dec; c->M = cfg->n_mode_ra; c->N = cfg->n_mode_dec;
    c->NG = cfg->n_gain_modes; c->npix = c->R * c->D; c->nk = c->M * c->N;
    c->B = c->A * (c->A - 1) / 2;
    c->prec = cfg->precision;
    c->rsz = c->prec == FM_PREC_FP64_SIMT ? 8 : 4;
    c->K = cfg->n_freq_modes;
    c->n_sky_m = (int64_t)c->F * c->nk;
    c->n_sky = c->K > 0 ? (int64_t)c->K * c->nk : c->n_sky_m;
    c->n_par = c->n_sky + 2LL * c->A * c->NG;
    c->n_vis = (int64_t)c->F * c->T * c->B;
    c->ant.assign(cfg->ant_enu_m, cfg->ant_enu_m + 3 * (size_t)c->A);
    c->freq.assign(cfg->freq_hz, cfg->freq_hz + c->F);
    c->lst.assign(cfg->lst_rad, cfg->lst_rad + c->T);
    c->cfg.ant_enu_m = c->ant.data();
    c->cfg.freq_hz = c->freq.data();
    c->cfg.lst_rad = c->lst.data();

    DevGeom &g = c->g;
    memset(&g, 0, sizeof(g));
    g.A = c->A; g.F = c->F; g.T = c->T; g.R = c->R; g.D = c->D; g.M = c->M; g.N = c->N; g.NG = c->NG;
    g.npix = c->npix; g.nk = c->nk; g.B = c->B; g.apad = (c->A + 3) / 4 * 4;
    g.inv_sigma2 = 1.0 / (cfg->sigma_noise * cfg->sigma_noise);
    size_t tp = (size_t)c->T * c->npix;
    double *d64;
    float *d32;
    FM_TRY(dalloc(*c, &d64, 3 * tp)); g.s64 = d64;
    FM_TRY(dalloc(*c, &d32, 6 * tp)); g.s32 = d32;
    FM_TRY(dalloc(*c, &d64, tp)); g.za2_64 = d64;
    FM_TRY(dalloc(*c, &d32, tp)); g.za2_32 = d32;
    FM_TRY(dalloc(*c, &d64, c->D)); g.domega64 = d64;
    FM_TRY(dalloc(*c, &d32, c->D)); g.domega32 = d32;
    FM_TRY(dalloc(*c, &d64, (size_t)c->R * c->M)); g.phi64 = d64;
    FM_TRY(dalloc(*c, &d32, (size_t)c->R * c->M)); g.phi32 = d32;
    FM_TRY(dalloc(*c, &d64, (size_t)c->D * c->N)); g.leg64 = d64;
    FM_TRY(dalloc(*c, &d32, (size_t)c->D * c->N)); g.leg32 = d32;
    FM_TRY(dalloc(*c, &d64, (size_t)c->F * c->NG)); g.gleg64 = d64;
    FM_TRY(dalloc(*c, &d32, (size_t)c->F * c->NG)); g.gleg32 = d32;
    FM_TRY(dalloc(*c, &d64, (size_t)c->F * c->A * 3)); g.kap64 = d64;
    FM_TRY(dalloc(*c, &d32, (size_t)c->F * c->A * 6)); g.kap32 = d32;
    FM_TRY(dalloc(*c, &d64, c->F)); g.bcoef64 = d64;
    if (cfg->beam_type == FM_BEAM_AIRY) {
        g.dish_ew = cfg->dish_ew_m;
        g.dish_ns = cfg->dish_ns_m;
        const size_t nb = (size_t)c->F * tp;
        FM_TRY(dalloc(*c, &d32, nb)); g.beam32 = d32;
        // FP64 table: kept by FP64 handles; FP32 handles use it once, for the FP64 monopole
        // visibilities at create time, and free it afterwards
        if (c->prec == FM_PREC_FP64_SIMT) { FM_TRY(dalloc(*c, &d64, nb)); g.beam64 = d64; }
        else {
            void *b = nullptr;
            FM_CK(cudaMalloc(&b, sizeof(double) * nb));
            g.beam64 = static_cast<double *>(b);
        }
    }
    FM_TRY(dalloc(*c, &d32, c->F)); g.bcoef32 = d32;
    FM_TRY(dalloc(*c, &d32, (size_t)c->npix)); g.dompix32 = d32;
    int *bl;
    FM_TRY(dalloc(*c, &bl, 2 * (size_t)c->B));
    std::vector<int> hb(2 * (size_t)c->B);
    for (int i = 0, b = 0; i < c->A; ++i)
        for (int j = i + 1; j < c->A; ++j, ++b) { hb[b] = i; hb[c->B + b] = j; }
    FM_CK(cudaMemcpy(bl, hb.data(), sizeof(int) * hb.size(), cudaMemcpyHostToDevice));
    g.bl_i = bl; g.bl_j = bl + c->B;
    FM_TRY(dalloc(*c, &c->status, 1));
    FM_CK(cudaMemset(c->status, 0, sizeof(int)));
    FM_TRY(dalloc(*c, &c->ticket, 1));
    FM_CK(cudaMemset(c->ticket, 0, sizeof(unsigned)));
    g.status = c->status;
    {   // equal channel spacing enables the frequency recurrence of the phasors
        double dnu = c->F > 1 ? c->freq[1] - c->freq[0] : 0.0;
        bool uni = c->F > 1 && dnu > 0.0;
        for (int f = 1; f < c->F && uni; ++f)
            if (std::fabs((c->freq[f] - c->freq[f - 1]) - dnu) > 1e-9 * c->freq[f]) uni = false;
        std::vector<float> dk(3 * (size_t)c->A, 0.f);
        for (int i = 0; i < c->A; ++i) {
            double n2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double v = dnu * c->ant[3 * i + k] / kCLight;
                dk[3 * i + k] = (float)v;
                n2 += v * v;
            }
            // the step factor exp(-2 pi i dkap . s) is evaluated by a short series that
            // holds for phases up to 1/8 turn (|s| = 1)
            if (std::sqrt(n2) > 0.125) uni = false;
        }
        float *ddk;
        FM_TRY(dalloc(*c, &ddk, dk.size()));
        FM_CK(cudaMemcpy(ddk, dk.data(), sizeof(float) * dk.size(), cudaMemcpyHostToDevice));
        g.dkap32 = ddk;
        g.uniform_freq = uni ? 1 : 0;
        bool flat = true;
        for (int i = 0; i < c->A; ++i)
            if (c->ant[3 * i + 2] != 0.0) flat = false;
        g.flat_array = flat ? 1 : 0;
    }

    size_t rs = c->rsz;
    FM_TRY(dalloc_bytes(*c, &c->data, (size_t)c->n_vis * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->mu, (size_t)c->n_par * rs));
    FM_TRY(dalloc_bytes(*c, &c->lam, (size_t)c->n_par * rs));
    size_t fp = (size_t)c->F * c->npix * rs;
    FM_TRY(dalloc_bytes(*c, &c->x, fp));
    FM_TRY(dalloc_bytes(*c, &c->xv, fp));
    FM_TRY(dalloc_bytes(*c, &c->xbar, fp));
    FM_TRY(dalloc_bytes(*c, &c->tmp, (size_t)c->F * c->R * c->N * rs));
    FM_TRY(dalloc_bytes(*c, &c->vis, (size_t)c->n_vis * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->dvis, (size_t)c->n_vis * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->omega, (size_t)c->n_vis * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->zpart, (size_t)c->F * c->T * c->A * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->gains, (size_t)c->F * c->A * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->dgains, (size_t)c->F * c->A * 2 * rs));
    FM_TRY(dalloc_bytes(*c, &c->work_par, (size_t)c->n_par * rs));
    FM_TRY(dalloc(*c, &c->chi2p, (size_t)c->F * c->T));
    FM_TRY(dalloc(*c, &c->red, 1024));
    FM_TRY(dalloc(*c, &c->scal, 64));
    FM_TRY(dalloc(*c, &c->tc_scale, (size_t)c->F));
    {
        double dra = (cfg->ra_max - cfg->ra_min) / c->R, ddec = (cfg->dec_max - cfg->dec_min) / c->D, mx = 0.0;
        for (int d = 0; d < c->D; ++d) {
            double w = dra * (std::sin(cfg->dec_min + (d + 1) * ddec) - std::sin(cfg->dec_min + d * ddec));
            if (w > mx) mx = w;
        }
        c->domega_max = (float)mx;
    }

    FM_TRY(launch_precompute(*c, 0));
    FM_CK(cudaStreamSynchronize(0));
    FM_TRY(freq_basis_setup(*c));
    FM_TRY(ha_setup(*c));
    if (c->prec != FM_PREC_FP64_SIMT) {
        // monopole split: U = V(x = 1) once, in FP64, stored as FP32 (through the hour-angle
        // geometry when that form is on: one sum per fringe group; else the direct FP64 sum)
        c->dc_split = true;
        FM_TRY(dalloc(*c, &c->dc_u, (size_t)c->n_vis * 2));
        FM_TRY(dalloc_bytes(*c, &c->dc_mean, (size_t)c->F * sizeof(float)));
        const fm_status hs = ha_monopole(*c, c->dc_u, 0);
        if (hs != FM_OK && hs != FM_ERR_UNSUPPORTED) return hs;
        if (hs == FM_ERR_UNSUPPORTED) {
            double *ones = nullptr, *u64 = nullptr;
            FM_CK(cudaMalloc(&ones, sizeof(double) * (size_t)c->F * c->npix));
            cudaError_t e = cudaMalloc(&u64, sizeof(double) * 2 * (size_t)c->n_vis);
            if (e != cudaSuccess) { cudaFree(ones); return cuda_fail(e, "cudaMalloc(U)", __FILE__, __LINE__); }
            std::vector<double> h1((size_t)c->F * c->npix, 1.0);
            fm_status s = FM_OK;
            if (cudaMemcpy(ones, h1.data(), sizeof(double) * h1.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                s = FM_ERR_CUDA;
            if (s == FM_OK) s = launch_vis<double>(*c, ones, u64, 0);
            if (s == FM_OK) s = launch_d2f(2 * c->n_vis, u64, c->dc_u, 0);
            cudaError_t e2 = cudaStreamSynchronize(0);
            cudaFree(ones);
            cudaFree(u64);
            if (s != FM_OK) return s;
            FM_CK(e2);
        }
        if (c->g.beam64) {                      // the FP64 beam table of an FP32 handle
            FM_CK(cudaDeviceSynchronize());
            cudaFree(const_cast<double *>(c->g.beam64));
            c->g.beam64 = nullptr;
        }
    }
    FM_TRY(modes_tc_setup(*c));
    return FM_OK;
}

// ------------------------------------------------------------------ drivers
// x -> V; with dc != nullptr the monopole visibilities dc[f * dcs] U[f][t][b] are added
// (inside the last kernel of the hour-angle form, as a separate pass otherwise)
template <typename R>
static fm_status run_vis(Ctx &c, const R *x, R *vis, cudaStream_t st, const R *dc = nullptr, long long dcs = 0,
                         bool xmax_ready = false, bool strips_ready = false, bool partials_only = false)
{
    // the tensor-core launchers time their main kernel themselves
    if constexpr (std::is_same<R, float>::value) {
        if (c.ha.on) return launch_vis_ha(c, x, vis, st, dc, dcs, xmax_ready, strips_ready, partials_only);
        if (c.prec >= FM_PREC_BF16X1) {
            FM_TRY(launch_vis_tc(c, x, vis, st));
            return dc ? launch_add_dc<R>(c, dc, dcs, vis, st) : FM_OK;
        }
    }
    FM_TRY(profiled(c, 0, st, [&]() -> fm_status { return launch_vis<R>(c, x, vis, st); }));
    return dc ? launch_add_dc<R>(c, dc, dcs, vis, st) : FM_OK;
}

template <typename R>
static fm_status run_adjoint(Ctx &c, const R *omega, R *xbar, cudaStream_t st, bool q_ready = false)
{
    if constexpr (std::is_same<R, float>::value) {
        if (c.ha.on) return launch_adjoint_ha(c, omega, xbar, st, q_ready);
        if (c.prec >= FM_PREC_BF16X1) return launch_adjoint_tc(c, omega, xbar, st);
    }
    return profiled(c, 1, st, [&]() -> fm_status { return launch_adjoint<R>(c, omega, xbar, st); });
}

template <typename R>
fm_status vis_of_modes(Ctx &c, const R *a, R *xbuf, R *vis, cudaStream_t st, bool partials_only)
{
    if (partials_only && !(std::is_same<R, float>::value && c.ha.on)) {
        set_error("unfinished visibilities exist only in the hour-angle form");
        return FM_ERR_STATE;
    }
    // hour-angle form after the tensor-core transform: the transform forms the channel maxima
    // of x that scale the sky strip, and with one CTA per channel the strips themselves
    unsigned *xmax = nullptr;
    StripArgs sa;
    bool strips = false;
    if constexpr (std::is_same<R, float>::value)
        if (c.ha.on && c.mtc.on) {
            strips = ha_strip_args(c, sa);
            if (!strips) FM_CK(cudaMemsetAsync(c.ha.xmax, 0, sizeof(unsigned) * c.F, st));
            xmax = c.ha.xmax;
        }
    const bool dc = c.dc_split;
    FM_TRY(launch_modes_forward<R>(c, a, xbuf, st, dc ? 1 : 0, xmax, strips ? &sa : nullptr));
    return run_vis<R>(c, xbuf, vis, st, dc ? a : nullptr, dc ? c.nk : 0, xmax != nullptr, strips, partials_only);
}
template fm_status vis_of_modes<float>(Ctx &, const float *, float *, float *, cudaStream_t, bool);
template fm_status vis_of_modes<double>(Ctx &, const double *, double *, double *, cudaStream_t, bool);

template <typename R>
fm_status run_chi2_grad(Ctx &c, const R *theta, double *chi2_out, double *u_out, R *grad, cudaStream_t st,
                        R *kick_p, const double *kick_prm, double kick_frac)
{
    if (!c.have_data) { set_error("fm_set_data has not been called"); return FM_ERR_STATE; }
    R *x = (R *)c.x, *vis = (R *)c.vis, *om = (R *)c.omega, *zp = (R *)c.zpart;
    const R *sky = theta;
    if (c.K > 0) {                          // Legendre-in-frequency coefficients -> channel modes
        FM_TRY(launch_freq_expand<R>(c, theta, (R *)c.ax, st));
        sky = (const R *)c.ax;
    }
    // hour-angle form: the epilogue forms the group sums of omega itself, and without the
    // delay filter (one LST pass) also V from the forward's partial sums
    const bool groups = std::is_same<R, float>::value && c.ha.on;
    HaVSrc hv;
    bool fused = false;
    if constexpr (std::is_same<R, float>::value)
        if (groups && !c.df_on) fused = ha_vsrc(c, c.dc_split ? sky : nullptr, c.nk, hv);
    FM_TRY(vis_of_modes<R>(c, sky, x, vis, st, fused));
    if (fused) {
        FM_TRY(launch_chi2_chan<R>(c, nullptr, theta + c.n_sky, om, zp, c.chi2p, groups, st, nullptr, &hv));
    } else if (c.df_on) {
        // delay filter: the filtered chi^2 and the residual weights sigma^2 F^T W F r, which the
        // epilogue then uses in place of m - d (its own chi^2 partials are not used)
        FM_TRY(launch_delay_filter<R>(c, vis, theta + c.n_sky, st));
        FM_TRY(launch_chi2_chan<R>(c, vis, theta + c.n_sky, om, zp, c.chi2p, groups, st, (const R *)c.df_r));
    } else {
        FM_TRY(launch_chi2_chan<R>(c, vis, theta + c.n_sky, om, zp, c.chi2p, groups, st));   // gains formed inside
    }
    FM_TRY(run_adjoint<R>(c, om, (R *)c.xbar, st, groups));
    FM_TRY(launch_modes_adjoint<R>(c, (R *)c.xbar, c.K > 0 ? (R *)c.gx : grad, st));
    if (c.K > 0) FM_TRY(launch_freq_contract<R>(c, (const R *)c.gx, grad, st));
    FM_TRY(launch_gain_reduce_chan<R>(c, zp, grad + c.n_sky, st));
    if (c.df_on)
        return launch_prior_and_total<R>(c, theta, grad, c.df_chi2p, c.df_nparts, chi2_out, u_out, st, kick_p,
                                         kick_prm, kick_frac);
    return launch_prior_and_total<R>(c, theta, grad, c.chi2p, c.F * c.T, chi2_out, u_out, st, kick_p, kick_prm,
                                     kick_frac);
}

template <typename R>
static fm_status run_hvp(Ctx &c, const R *theta, const R *v, R *hv, int full, cudaStream_t st)
{
    if (!c.have_data) { set_error("fm_set_data has not been called"); return FM_ERR_STATE; }
    if (c.df_on) { set_error("Hessian-vector products with the delay filter are not implemented"); return FM_ERR_UNSUPPORTED; }
    R *x = (R *)c.x, *xv = (R *)c.xv;
    FM_TRY(launch_gains<R>(c, theta + c.n_sky, (R *)c.gains, st));
    FM_TRY(launch_gains<R>(c, v + c.n_sky, (R *)c.dgains, st));
    const R *sky = theta, *vsky = v;
    if (c.K > 0) {
        FM_TRY(launch_freq_expand<R>(c, theta, (R *)c.ax, st));
        FM_TRY(launch_freq_expand<R>(c, v, (R *)c.avx, st));
        sky = (const R *)c.ax;
        vsky = (const R *)c.avx;
    }
    FM_TRY(vis_of_modes<R>(c, sky, x, (R *)c.vis, st));
    FM_TRY(vis_of_modes<R>(c, vsky, xv, (R *)c.dvis, st));
    FM_TRY(launch_hvp_mid<R>(c, (R *)c.vis, (R *)c.dvis, (R *)c.gains, (R *)c.dgains, full, (R *)c.omega,
                             (R *)c.zpart, st));
    FM_TRY(run_adjoint<R>(c, (R *)c.omega, (R *)c.xbar, st));
    FM_TRY(launch_modes_adjoint<R>(c, (R *)c.xbar, c.K > 0 ? (R *)c.gx : hv, st));
    if (c.K > 0) FM_TRY(launch_freq_contract<R>(c, (const R *)c.gx, hv, st));
    FM_TRY(launch_gain_reduce<R>(c, (R *)c.zpart, hv + c.n_sky, st));
    return launch_prior_hvp<R>(c, v, hv, st);
}

template fm_status run_chi2_grad<float>(Ctx &, const float *, double *, double *, float *, cudaStream_t, float *,
                                        const double *, double);
template fm_status run_chi2_grad<double>(Ctx &, const double *, double *, double *, double *, cudaStream_t, double *,
                                         const double *, double);

}  // namespace fm

using namespace fm;

#define FM_HANDLE_OK(h)                                                   \
    do {                                                                  \
        if (!(h)) return invalid("handle is NULL");                       \
    } while (0)

extern "C" {

const char *fm_last_error(void) { return g_err; }

fm_status fm_create(const fm_config *cfg, fm_handle *out)
{
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    FM_TRY(validate(cfg));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        set_error("no CUDA device is visible");
        return FM_ERR_CUDA;
    }
    Ctx *c = new Ctx();
    fm_status s = create_impl(cfg, c);
    if (s != FM_OK) {
        free_ctx(c);
        return s;
    }
    *out = reinterpret_cast<fm_handle>(c);
    return FM_OK;
}

fm_status fm_destroy(fm_handle h)
{
    if (!h) return FM_OK;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    cudaDeviceSynchronize();
    free_ctx(c);
    return FM_OK;
}

int64_t fm_num_params(fm_handle h) { return h ? reinterpret_cast<Ctx *>(h)->n_par : -1; }
int64_t fm_num_vis(fm_handle h) { return h ? reinterpret_cast<Ctx *>(h)->n_vis : -1; }

fm_status fm_set_data(fm_handle h, const void *dev_vis, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_vis) return invalid("dev_vis is NULL");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    FM_CK(cudaMemcpyAsync(c.data, dev_vis, (size_t)c.n_vis * 2 * c.rsz, cudaMemcpyDeviceToDevice, stream));
    c.have_data = true;
    return FM_OK;
}

fm_status fm_set_prior(fm_handle h, const void *dev_mu, const void *dev_inv_var, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_mu || !dev_inv_var) return invalid("prior arrays are NULL");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    FM_CK(cudaMemcpyAsync(c.mu, dev_mu, (size_t)c.n_par * c.rsz, cudaMemcpyDeviceToDevice, stream));
    FM_CK(cudaMemcpyAsync(c.lam, dev_inv_var, (size_t)c.n_par * c.rsz, cudaMemcpyDeviceToDevice, stream));
    c.have_prior = true;
    return FM_OK;
}

fm_status fm_forward(fm_handle h, const void *dev_theta, void *dev_vis_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_theta || !dev_vis_out) return invalid("NULL device pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (c.prec == FM_PREC_FP64_SIMT) {
        const double *th = (const double *)dev_theta, *sky = th;
        if (c.K > 0) {
            FM_TRY(launch_freq_expand<double>(c, th, (double *)c.ax, stream));
            sky = (const double *)c.ax;
        }
        FM_TRY(launch_gains<double>(c, th + c.n_sky, (double *)c.gains, stream));
        FM_TRY(vis_of_modes<double>(c, sky, (double *)c.x, (double *)c.vis, stream));
        return launch_apply_gains<double>(c, (double *)c.vis, (double *)c.gains, (double *)dev_vis_out, stream);
    }
    const float *th = (const float *)dev_theta, *sky = th;
    if (c.K > 0) {
        FM_TRY(launch_freq_expand<float>(c, th, (float *)c.ax, stream));
        sky = (const float *)c.ax;
    }
    FM_TRY(launch_gains<float>(c, th + c.n_sky, (float *)c.gains, stream));
    FM_TRY(vis_of_modes<float>(c, sky, (float *)c.x, (float *)c.vis, stream));
    return launch_apply_gains<float>(c, (float *)c.vis, (float *)c.gains, (float *)dev_vis_out, stream);
}

fm_status fm_forward_pixels(fm_handle h, const void *dev_x, void *dev_vis_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_x || !dev_vis_out) return invalid("NULL device pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (c.prec == FM_PREC_FP64_SIMT) return run_vis<double>(c, (const double *)dev_x, (double *)dev_vis_out, stream);
    if (c.dc_split) {
        FM_TRY(launch_center<float>(c, (const float *)dev_x, (float *)c.x, (float *)c.dc_mean, stream));
        return run_vis<float>(c, (const float *)c.x, (float *)dev_vis_out, stream, (const float *)c.dc_mean, 1);
    }
    return run_vis<float>(c, (const float *)dev_x, (float *)dev_vis_out, stream);
}

fm_status fm_sky_pixels(fm_handle h, const void *dev_theta, void *dev_x_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_theta || !dev_x_out) return invalid("NULL device pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (c.prec == FM_PREC_FP64_SIMT) {
        const double *sky = (const double *)dev_theta;
        if (c.K > 0) {
            FM_TRY(launch_freq_expand<double>(c, sky, (double *)c.ax, stream));
            sky = (const double *)c.ax;
        }
        return launch_modes_forward<double>(c, sky, (double *)dev_x_out, stream, 0);
    }
    const float *sky = (const float *)dev_theta;
    if (c.K > 0) {
        FM_TRY(launch_freq_expand<float>(c, sky, (float *)c.ax, stream));
        sky = (const float *)c.ax;
    }
    return launch_modes_forward<float>(c, sky, (float *)dev_x_out, stream, 0);
}

fm_status fm_chi2_grad(fm_handle h, const void *dev_theta, double *dev_chi2_out, double *dev_u_out,
                       void *dev_grad_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_theta || !dev_chi2_out || !dev_grad_out) return invalid("NULL device pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (c.prec == FM_PREC_FP64_SIMT)
        return run_chi2_grad<double>(c, (const double *)dev_theta, dev_chi2_out, dev_u_out, (double *)dev_grad_out,
                                     stream);
    return run_chi2_grad<float>(c, (const float *)dev_theta, dev_chi2_out, dev_u_out, (float *)dev_grad_out, stream);
}

fm_status fm_hvp(fm_handle h, const void *dev_theta, const void *dev_v, void *dev_hv_out, int full, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_theta || !dev_v || !dev_hv_out) return invalid("NULL device pointer");
    if (full != 0 && full != 1) return invalid("full must be 0 or 1");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (c.prec == FM_PREC_FP64_SIMT)
        return run_hvp<double>(c, (const double *)dev_theta, (const double *)dev_v, (double *)dev_hv_out, full, stream);
    return run_hvp<float>(c, (const float *)dev_theta, (const float *)dev_v, (float *)dev_hv_out, full, stream);
}

fm_status fm_build_precond(fm_handle h, const void *dev_theta, int block, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_theta) return invalid("NULL device pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (block != 1 && block != 64) return invalid("block must be 1 or 64");
    if (c.nk % block != 0) return invalid("n_mode_ra*n_mode_dec must be a multiple of block");
    if (!c.have_data) { set_error("fm_set_data has not been called"); return FM_ERR_STATE; }
    if (c.prec == FM_PREC_FP64_SIMT) return run_build_precond<double>(c, (const double *)dev_theta, block, stream);
    return run_build_precond<float>(c, (const float *)dev_theta, block, stream);
}

int64_t fm_precond_size(fm_handle h)
{
    if (!h) return -1;
    return reinterpret_cast<Ctx *>(h)->pc_size;
}

fm_status fm_get_precond_blocks(fm_handle h, double *dev_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_out) return invalid("NULL device pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (!c.pc_blocks) { set_error("fm_build_precond has not been called"); return FM_ERR_STATE; }
    FM_CK(cudaMemcpyAsync(dev_out, c.pc_blocks, sizeof(double) * (size_t)c.pc_size, cudaMemcpyDeviceToDevice, stream));
    return FM_OK;
}

fm_status fm_leapfrog(fm_handle h, void *dev_q, void *dev_p, double eps, int n_steps, double u_accept,
                      double *dev_h_out, int *dev_accepted_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_q || !dev_p || !dev_h_out || !dev_accepted_out) return invalid("NULL device pointer");
    if (!(eps > 0.0) || !std::isfinite(eps)) return invalid("eps must be > 0");
    if (n_steps < 1 || n_steps > 100000) return invalid("n_steps must be in [1, 100000]");
    if (!(u_accept >= 0.0 && u_accept < 1.0)) return invalid("u_accept must be in [0, 1)");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (!c.have_data) { set_error("fm_set_data has not been called"); return FM_ERR_STATE; }
    if (!c.pc_chol) { set_error("fm_build_precond has not been called"); return FM_ERR_STATE; }
    if (c.prec == FM_PREC_FP64_SIMT) {
        FM_TRY(set_leapfrog_params<double>(c, eps, u_accept, stream));
        return run_leapfrog<double>(c, (double *)dev_q, (double *)dev_p, c.lf_prm, n_steps, dev_h_out,
                                    dev_accepted_out, stream);
    }
    FM_TRY(set_leapfrog_params<float>(c, eps, u_accept, stream));
    return run_leapfrog<float>(c, (float *)dev_q, (float *)dev_p, c.lf_prm, n_steps, dev_h_out, dev_accepted_out,
                               stream);
}

fm_status fm_precond_apply(fm_handle h, int op, const void *dev_in, void *dev_out, fm_stream stream)
{
    FM_HANDLE_OK(h);
    if (!dev_in || !dev_out) return invalid("NULL device pointer");
    if (dev_in == dev_out) return invalid("in and out may not alias");
    if (op < 0 || op > 3) return invalid("op must be 0..3");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (!c.pc_chol) { set_error("fm_build_precond has not been called"); return FM_ERR_STATE; }
    if (c.prec == FM_PREC_FP64_SIMT)
        return run_precond_apply<double>(c, op, (const double *)dev_in, (double *)dev_out, stream);
    return run_precond_apply<float>(c, op, (const float *)dev_in, (float *)dev_out, stream);
}

fm_status fm_set_profiling(fm_handle h, int on)
{
    FM_HANDLE_OK(h);
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    c.prof_on = on != 0;
    return FM_OK;
}

fm_status fm_get_profile(fm_handle h, double *out_ms, int64_t *out_count)
{
    FM_HANDLE_OK(h);
    if (!out_ms || !out_count) return invalid("NULL output pointer");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    double ms[2] = {0.0, 0.0};
    int64_t cnt[2] = {0, 0};
    for (auto &r : c.prof_rec) {
        FM_CK(cudaEventSynchronize(r.second.second));
        float t = 0.f;
        FM_CK(cudaEventElapsedTime(&t, r.second.first, r.second.second));
        ms[r.first] += t;
        cnt[r.first] += 1;
    }
    c.prof_rec.clear();
    c.prof_next = 0;
    for (int k = 0; k < 2; ++k) { out_ms[k] = ms[k]; out_count[k] = cnt[k]; }
    return FM_OK;
}

fm_status fm_contraction_info(fm_handle h, int32_t *out)
{
    FM_HANDLE_OK(h);
    if (!out) return invalid("out is NULL");
    const Ctx &c = *reinterpret_cast<const Ctx *>(h);
    out[0] = c.ha.on ? 2 : (c.prec >= FM_PREC_BF16X1 ? 1 : 0);
    out[1] = c.ha.on ? c.ha.U : c.B;
    out[2] = c.ha.on ? c.ha.k : 0;
    out[3] = c.ha.on ? c.ha.nhp : 0;
    return FM_OK;
}

int64_t fm_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

fm_status fm_sync_status(fm_handle h, fm_stream stream)
{
    FM_HANDLE_OK(h);
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    FM_CK(cudaStreamSynchronize(stream));
    int s = 0;
    FM_CK(cudaMemcpy(&s, c.status, sizeof(int), cudaMemcpyDeviceToHost));
    FM_CK(cudaMemset(c.status, 0, sizeof(int)));
    if (s != 0) {
        set_error("device status: %s", s == FM_ERR_NONFINITE ? "non-finite chi^2 or Hamiltonian"
                                     : s == FM_ERR_TIMEOUT   ? "device wait timed out"
                                                             : "error");
        return (fm_status)s;
    }
    return FM_OK;
}

}  // extern "C"
