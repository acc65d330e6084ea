/*
 * fm_oracle.c -- plain, slow, FP64 CPU reference of the visibility forward model
 * of arXiv:2504.07090 (Kern, "A Differentiable, End-to-End Forward Model for 21 cm
 * Cosmology").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: it exists so the tests, the smoke check and the CPU-baseline leg of the
 * benchmark can compare the CUDA library against the paper's definitions.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes, term by term, with no factorisation:
 *   - pixel centres, exact cell solid angles and topocentric directions of a regular
 *     RA x Dec grid (Sec. 2.1, discretised RIME, Eq. rime_discrete; grid of Sec. 3.2);
 *   - the separable cos/sin(RA) x Legendre(Dec) mode basis evaluated pixel by pixel
 *     (Eq. fg_separable, Eq. eor_model; azimuthal periodicity of App. A.2);
 *   - the primary beam (total-power response A of Eq. rime_integral): a Gaussian in zenith
 *     angle, or the modified Airy pattern of Eq. airy squared, with J1 from Bessel's integral;
 *   - V_pq(nu,t) = sum_j dOmega_j A_j K_jpq B_j with K = exp(-2 pi i b_pq . s nu / c),
 *     b_pq = r_p - r_q, one baseline at a time (Eq. rime_integral, Eq. rime_discrete);
 *   - its adjoint with respect to the pixel values, baseline by baseline.
 * Everything is double precision with libm cos/sin; OpenMP only splits independent
 * outputs, so every sum is taken in one fixed order and results are bitwise
 * reproducible for any thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C_LIGHT 299792458.0
#define ORC_PI 3.14159265358979323846

typedef struct {
    int n_ant, n_freq, n_lst;
    int n_ra, n_dec, n_mode_ra, n_mode_dec, n_gain;
    const double *ant_enu;   /* [n_ant][3] metres */
    const double *freq_hz;   /* [n_freq] */
    const double *lst_rad;   /* [n_lst] */
    double lat_rad, ra_min, ra_max, dec_min, dec_max;
    double beam_fwhm_ref_rad, beam_ref_hz;  /* fwhm <= 0: isotropic above the horizon */
    int beam_type;                          /* 0 Gaussian, 1 Airy (Eq. airy) */
    double dish_ew, dish_ns;                /* Airy aperture diameters (m) */
} orc_problem;

typedef struct {
    orc_problem P;
    int n_pix, n_bl;
    double *ant, *freq, *lst;
    int *bl_i, *bl_j;        /* baseline b = (i<j), row-major over i then j */
    double *ra_c, *dec_c;    /* cell centres */
    double *domega;          /* [n_dec] cell solid angle (same for every RA cell of a row) */
    double *phi;             /* [n_ra][n_mode_ra]  RA basis */
    double *leg;             /* [n_dec][n_mode_dec] Dec basis */
    double *s;               /* [n_lst][n_pix][3]  topocentric east, north, up */
    double *gleg;            /* [n_freq][n_gain] Legendre of the normalised frequency */
} orc_geom;

static void orc_legendre(double x, int n, double *out)
{
    /* Bonnet's three-term recursion for P_0 .. P_{n-1}. */
    if (n <= 0) return;
    out[0] = 1.0;
    if (n == 1) return;
    out[1] = x;
    for (int k = 1; k + 1 < n; ++k)
        out[k + 1] = ((2.0 * k + 1.0) * x * out[k] - (double)k * out[k - 1]) / (k + 1.0);
}

static double orc_ra_function(int m, int n_mode_ra, double ahat)
{
    /* 1, cos(k a), sin(k a) for k = 1 .. M/2-1, and cos(M/2 a) last: M functions that
     * are periodic over the RA span (azimuthal condition of App. A.2). */
    if (m == 0) return 1.0;
    if (m == n_mode_ra - 1 && n_mode_ra >= 2) return cos(0.5 * n_mode_ra * ahat);
    int k = (m + 1) / 2;
    return (m % 2 == 1) ? cos(k * ahat) : sin(k * ahat);
}

orc_geom *orc_create(const orc_problem *in)
{
    orc_geom *G = (orc_geom *)calloc(1, sizeof(orc_geom));
    if (!G) return NULL;
    G->P = *in;
    const orc_problem *P = &G->P;
    int A = P->n_ant, F = P->n_freq, T = P->n_lst;
    G->n_pix = P->n_ra * P->n_dec;
    G->n_bl = A * (A - 1) / 2;
    G->ant = (double *)malloc(sizeof(double) * 3 * (size_t)A);
    G->freq = (double *)malloc(sizeof(double) * (size_t)F);
    G->lst = (double *)malloc(sizeof(double) * (size_t)T);
    memcpy(G->ant, in->ant_enu, sizeof(double) * 3 * (size_t)A);
    memcpy(G->freq, in->freq_hz, sizeof(double) * (size_t)F);
    memcpy(G->lst, in->lst_rad, sizeof(double) * (size_t)T);
    G->P.ant_enu = G->ant;
    G->P.freq_hz = G->freq;
    G->P.lst_rad = G->lst;

    G->bl_i = (int *)malloc(sizeof(int) * (size_t)(G->n_bl > 0 ? G->n_bl : 1));
    G->bl_j = (int *)malloc(sizeof(int) * (size_t)(G->n_bl > 0 ? G->n_bl : 1));
    int b = 0;
    for (int i = 0; i < A; ++i)
        for (int j = i + 1; j < A; ++j) { G->bl_i[b] = i; G->bl_j[b] = j; ++b; }

    int R = P->n_ra, D = P->n_dec, M = P->n_mode_ra, N = P->n_mode_dec;
    double dra = (P->ra_max - P->ra_min) / R;
    double ddec = (P->dec_max - P->dec_min) / D;
    G->ra_c = (double *)malloc(sizeof(double) * (size_t)R);
    G->dec_c = (double *)malloc(sizeof(double) * (size_t)D);
    G->domega = (double *)malloc(sizeof(double) * (size_t)D);
    for (int r = 0; r < R; ++r) G->ra_c[r] = P->ra_min + (r + 0.5) * dra;
    for (int d = 0; d < D; ++d) {
        G->dec_c[d] = P->dec_min + (d + 0.5) * ddec;
        /* exact area of an RA x Dec cell: dRA * (sin dec_hi - sin dec_lo) */
        G->domega[d] = dra * (sin(P->dec_min + (d + 1) * ddec) - sin(P->dec_min + d * ddec));
    }

    G->phi = (double *)malloc(sizeof(double) * (size_t)R * (size_t)M);
    for (int r = 0; r < R; ++r) {
        double ahat = 2.0 * ORC_PI * (G->ra_c[r] - P->ra_min) / (P->ra_max - P->ra_min);
        for (int m = 0; m < M; ++m) G->phi[(size_t)r * M + m] = orc_ra_function(m, M, ahat);
    }
    G->leg = (double *)malloc(sizeof(double) * (size_t)D * (size_t)N);
    for (int d = 0; d < D; ++d) {
        double dhat = 2.0 * (G->dec_c[d] - P->dec_min) / (P->dec_max - P->dec_min) - 1.0;
        orc_legendre(dhat, N, G->leg + (size_t)d * N);
    }

    /* Topocentric unit vectors: hour angle H = LST - RA, standard equatorial to
     * east/north/up rotation at latitude lat. */
    size_t np_ = (size_t)G->n_pix;
    G->s = (double *)malloc(sizeof(double) * 3 * np_ * (size_t)T);
    double sl = sin(P->lat_rad), cl = cos(P->lat_rad);
    for (int t = 0; t < T; ++t)
        for (int d = 0; d < D; ++d)
            for (int r = 0; r < R; ++r) {
                double H = G->lst[t] - G->ra_c[r];
                double dec = G->dec_c[d];
                double *s = G->s + 3 * ((size_t)t * np_ + (size_t)d * R + r);
                s[0] = -cos(dec) * sin(H);
                s[1] = cl * sin(dec) - sl * cos(dec) * cos(H);
                s[2] = sl * sin(dec) + cl * cos(dec) * cos(H);
            }

    int NG = P->n_gain;
    G->gleg = (double *)malloc(sizeof(double) * (size_t)F * (size_t)(NG > 0 ? NG : 1));
    double fmin = G->freq[0], fmax = G->freq[0];
    for (int f = 1; f < F; ++f) {
        if (G->freq[f] < fmin) fmin = G->freq[f];
        if (G->freq[f] > fmax) fmax = G->freq[f];
    }
    for (int f = 0; f < F; ++f) {
        double nhat = (fmax > fmin) ? 2.0 * (G->freq[f] - fmin) / (fmax - fmin) - 1.0 : 0.0;
        orc_legendre(nhat, NG, G->gleg + (size_t)f * NG);
    }
    return G;
}

void orc_destroy(orc_geom *G)
{
    if (!G) return;
    free(G->ant); free(G->freq); free(G->lst); free(G->bl_i); free(G->bl_j);
    free(G->ra_c); free(G->dec_c); free(G->domega); free(G->phi); free(G->leg);
    free(G->s); free(G->gleg); free(G);
}

void orc_get_geometry(const orc_geom *G, double *ra_c, double *dec_c, double *domega,
                      double *phi, double *leg, double *s, double *gleg)
{
    const orc_problem *P = &G->P;
    if (ra_c) memcpy(ra_c, G->ra_c, sizeof(double) * (size_t)P->n_ra);
    if (dec_c) memcpy(dec_c, G->dec_c, sizeof(double) * (size_t)P->n_dec);
    if (domega) memcpy(domega, G->domega, sizeof(double) * (size_t)P->n_dec);
    if (phi) memcpy(phi, G->phi, sizeof(double) * (size_t)P->n_ra * P->n_mode_ra);
    if (leg) memcpy(leg, G->leg, sizeof(double) * (size_t)P->n_dec * P->n_mode_dec);
    if (s) memcpy(s, G->s, sizeof(double) * 3 * (size_t)G->n_pix * P->n_lst);
    if (gleg) memcpy(gleg, G->gleg, sizeof(double) * (size_t)P->n_freq * P->n_gain);
}

double orc_bessel_j1(double x)
{
    /* Bessel's integral J1(x) = (1 / 2 pi) int_0^2pi cos(tau - x sin tau) d tau, by the
     * trapezoidal rule over the full period (exponentially convergent for this periodic,
     * analytic integrand; 2 |x| + 64 nodes). */
    int n = 2 * (int)fabs(x) + 64;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
        double tau = 2.0 * ORC_PI * k / n;
        acc += cos(tau - x * sin(tau));
    }
    return acc / n;
}

double orc_beam_dir(const orc_geom *G, double nu, double e, double n, double u)
{
    /* Total-power beam at unit direction (east, north, up).  Airy (Eq. airy): (2 J1(x) / x)^2,
     * x = D_eff sin(za) pi nu / c with D_eff = D_ns + sin^2(az) (D_ew - D_ns), the azimuth
     * measured from north through east (sin(az) = e / sqrt(e^2 + n^2)), sin(za) = sqrt(e^2 + n^2). */
    if (G->P.beam_type != 1) {
        extern double orc_beam(const orc_geom *G, double nu, double s_up);
        return orc_beam(G, nu, u);
    }
    if (u <= 0.0) return 0.0;
    double sinza = sqrt(e * e + n * n);
    if (sinza == 0.0) return 1.0;
    double sin2az = (e * e) / (sinza * sinza);
    double deff = G->P.dish_ns + sin2az * (G->P.dish_ew - G->P.dish_ns);
    double x = deff * sinza * ORC_PI * nu / ORC_C_LIGHT;
    double a;
    if (x < 0.1) {
        /* near the zenith the quotient J1(x) / x of an absolutely accurate J1 is not: the
         * series 2 J1(x) / x = sum_k (-1)^k (x / 2)^(2k) / (k! (k + 1)!) instead */
        double h2 = 0.25 * x * x, term = 1.0;
        a = 1.0;
        for (int k = 1; k < 8; ++k) {
            term *= -h2 / ((double)k * (k + 1));
            a += term;
        }
    } else {
        a = 2.0 * orc_bessel_j1(x) / x;
    }
    return a * a;
}

double orc_beam(const orc_geom *G, double nu, double s_up)
{
    /* Gaussian total-power beam in zenith angle, FWHM = fwhm_ref * ref_hz / nu, zero at
     * and below the horizon; fwhm_ref <= 0 selects an isotropic beam. */
    if (s_up <= 0.0) return 0.0;
    if (G->P.beam_fwhm_ref_rad <= 0.0) return 1.0;
    double za = acos(s_up > 1.0 ? 1.0 : s_up);
    double fwhm = G->P.beam_fwhm_ref_rad * G->P.beam_ref_hz / nu;
    double sig = fwhm / sqrt(8.0 * log(2.0));
    return exp(-za * za / (2.0 * sig * sig));
}

void orc_sky(const orc_geom *G, const double *a_f, double *x_f)
{
    /* x(pixel) = sum_{m,n} Phi_m(RA) P_n(Dec) a_{m n}: the dense double sum. */
    const orc_problem *P = &G->P;
    int R = P->n_ra, D = P->n_dec, M = P->n_mode_ra, N = P->n_mode_dec;
#pragma omp parallel for schedule(static)
    for (int p = 0; p < R * D; ++p) {
        int d = p / R, r = p % R;
        double acc = 0.0;
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n)
                acc += G->phi[(size_t)r * M + m] * G->leg[(size_t)d * N + n] * a_f[(size_t)m * N + n];
        x_f[p] = acc;
    }
}

void orc_sky_adjoint(const orc_geom *G, const double *xbar_f, double *abar_f)
{
    /* abar_{m n} = sum_pixels Phi_m(RA) P_n(Dec) xbar(pixel): transpose of orc_sky. */
    const orc_problem *P = &G->P;
    int R = P->n_ra, D = P->n_dec, M = P->n_mode_ra, N = P->n_mode_dec;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < M * N; ++k) {
        int m = k / N, n = k % N;
        double acc = 0.0;
        for (int d = 0; d < D; ++d)
            for (int r = 0; r < R; ++r)
                acc += G->phi[(size_t)r * M + m] * G->leg[(size_t)d * N + n] * xbar_f[(size_t)d * R + r];
        abar_f[k] = acc;
    }
}

static void orc_pixel_weights(const orc_geom *G, int f, int t, const double *x_f, double *w)
{
    /* w_j = dOmega_j A_j(nu) B_j for every pixel of channel f at LST t. */
    const orc_problem *P = &G->P;
    int R = P->n_ra;
    double nu = G->freq[f];
    const double *s = G->s + 3 * (size_t)t * G->n_pix;
    for (int p = 0; p < G->n_pix; ++p)
        w[p] = G->domega[p / R] * orc_beam_dir(G, nu, s[3 * p], s[3 * p + 1], s[3 * p + 2]) * (x_f ? x_f[p] : 1.0);
}

void orc_vis_ft(const orc_geom *G, int f, int t, const double *x_f, double *V)
{
    /* V_b = sum_j w_j exp(-2 pi i nu (r_i - r_j) . s_j / c), baseline by baseline. */
    int np_ = G->n_pix;
    double nu = G->freq[f];
    const double *s = G->s + 3 * (size_t)t * np_;
    double *w = (double *)malloc(sizeof(double) * (size_t)np_);
    orc_pixel_weights(G, f, t, x_f, w);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < G->n_bl; ++b) {
        const double *ri = G->ant + 3 * G->bl_i[b], *rj = G->ant + 3 * G->bl_j[b];
        double bx = ri[0] - rj[0], by = ri[1] - rj[1], bz = ri[2] - rj[2];
        double re = 0.0, im = 0.0;
        for (int p = 0; p < np_; ++p) {
            if (w[p] == 0.0) continue;
            double ph = -2.0 * ORC_PI * nu * (bx * s[3 * p] + by * s[3 * p + 1] + bz * s[3 * p + 2]) / ORC_C_LIGHT;
            re += w[p] * cos(ph);
            im += w[p] * sin(ph);
        }
        V[2 * b] = re;
        V[2 * b + 1] = im;
    }
    free(w);
}

void orc_vis_one(const orc_geom *G, int f, int t, int b, const double *x_f, double *V2)
{
    /* One visibility, same sum as orc_vis_ft (used for sampled checks at full size). */
    int np_ = G->n_pix, R = G->P.n_ra;
    double nu = G->freq[f];
    const double *s = G->s + 3 * (size_t)t * np_;
    const double *ri = G->ant + 3 * G->bl_i[b], *rj = G->ant + 3 * G->bl_j[b];
    double bx = ri[0] - rj[0], by = ri[1] - rj[1], bz = ri[2] - rj[2];
    double re = 0.0, im = 0.0;
    for (int p = 0; p < np_; ++p) {
        double w = G->domega[p / R] * orc_beam_dir(G, nu, s[3 * p], s[3 * p + 1], s[3 * p + 2]) * x_f[p];
        if (w == 0.0) continue;
        double ph = -2.0 * ORC_PI * nu * (bx * s[3 * p] + by * s[3 * p + 1] + bz * s[3 * p + 2]) / ORC_C_LIGHT;
        re += w * cos(ph);
        im += w * sin(ph);
    }
    V2[0] = re;
    V2[1] = im;
}

void orc_adjoint_ft(const orc_geom *G, int f, int t, const double *omega, double *xbar_f)
{
    /* xbar_j += dOmega_j A_j sum_b Re[conj(omega_b) K_bj]: the transpose of orc_vis_ft
     * with respect to the real pixel values (reverse-mode step of Sec. 2.3). */
    int np_ = G->n_pix, R = G->P.n_ra;
    double nu = G->freq[f];
    const double *s = G->s + 3 * (size_t)t * np_;
#pragma omp parallel for schedule(static)
    for (int p = 0; p < np_; ++p) {
        double w = G->domega[p / R] * orc_beam_dir(G, nu, s[3 * p], s[3 * p + 1], s[3 * p + 2]);
        if (w == 0.0) continue;
        double acc = 0.0;
        for (int b = 0; b < G->n_bl; ++b) {
            const double *ri = G->ant + 3 * G->bl_i[b], *rj = G->ant + 3 * G->bl_j[b];
            double ph = -2.0 * ORC_PI * nu * ((ri[0] - rj[0]) * s[3 * p] + (ri[1] - rj[1]) * s[3 * p + 1]
                                              + (ri[2] - rj[2]) * s[3 * p + 2]) / ORC_C_LIGHT;
            /* Re[conj(o) e^{i ph}] = o_re cos ph + o_im sin ph */
            acc += omega[2 * b] * cos(ph) + omega[2 * b + 1] * sin(ph);
        }
        xbar_f[p] += w * acc;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
