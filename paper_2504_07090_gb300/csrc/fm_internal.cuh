// Internal declarations of libfm: the handle, the device parameter block passed to
// every kernel, launch helpers and error plumbing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fm.h"

namespace fm {

constexpr double kCLight = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

// Everything a kernel needs to know about the problem, by value.
struct DevGeom {
    int A, F, T, R, D, M, N, NG, npix, nk, B;
    int apad;                 // antennas padded to a multiple of 4
    double inv_sigma2;        // 1 / sigma^2
    // FP64 precompute
    const double *s64;        // [T][npix][3] topocentric east, north, up
    const double *za2_64;     // [T][npix] squared zenith angle, < 0 below the horizon
    const double *domega64;   // [D]
    const double *phi64;      // [R][M]
    const double *leg64;      // [D][N]
    const double *gleg64;     // [F][NG]
    const double *kap64;      // [F][A][3]   nu r_i / c (turns per unit direction cosine)
    const double *bcoef64;    // [F]  beam exponent: A = exp(bcoef * za^2)
    // FP32 precompute
    const float *s32;         // [T][npix][6] two-float (hi, lo) east, north, up
    const float *za2_32;      // [T][npix]
    const float *domega32;    // [D]
    const float *phi32;       // [R][M]
    const float *leg32;       // [D][N]
    const float *gleg32;      // [F][NG]
    const float *kap32;       // [F][A][6] two-float
    const float *bcoef32;     // [F]
    const float *dompix32;    // [npix] cell solid angle of each pixel
    const float *dkap32;      // [A][3] channel step dnu * r_i / c (turns per unit direction cosine)
    int uniform_freq;         // channels equally spaced and |dkap| <= 1/8: E(nu + dnu) = E(nu) exp(-2 pi i dkap . s)
    int flat_array;           // every antenna has up = 0: phases need only east and north
    const int *bl_i, *bl_j;   // [B]
    int *status;              // device status word (fm_status codes)
    // Airy beam (Eq. airy): tables of the power beam per (channel, LST, pixel); NULL for the
    // Gaussian beam, which the kernels form from za2 and bcoef
    const float *beam32;      // [F][T][npix]
    const double *beam64;     // [F][T][npix] (FP64 handles)
    double dish_ew, dish_ns;  // metres
    const double *freq64;     // [F] channel frequencies (Hz)
};

// Bessel function of the first kind of order 1 in FP64: its power series
// sum_k (-1)^k (x/2)^(2k+1) / (k! (k+1)!) for |x| <= 12, and Hankel's asymptotic expansion
// J1(x) ~ sqrt(2 / (pi x)) (P cos w - Q sin w), w = x - 3 pi / 4, with
// P = sum_k (-1)^k a_2k / x^2k, Q = sum_k (-1)^k a_2k+1 / x^(2k+1),
// a_k = a_(k-1) (4 - (2k - 1)^2) / (8 k), a_0 = 1 (summed while the terms decrease) above.
__host__ __device__ inline double bessel_j1(double x)
{
    const double ax = x < 0.0 ? -x : x;
    double r;
    if (ax <= 12.0) {
        const double h = 0.5 * ax, h2 = h * h;
        double term = h, sum = h;
        for (int k = 1; k < 60; ++k) {
            term *= -h2 / ((double)k * (double)(k + 1));
            sum += term;
            if ((term < 0 ? -term : term) < 1e-18 * (sum < 0 ? -sum : sum)) break;
        }
        r = sum;
    } else {
        double p = 1.0, q = 0.0, a = 1.0, xp = 1.0, last = 1e300;
        for (int k = 1; k < 40; ++k) {
            a *= (4.0 - (double)(2 * k - 1) * (2 * k - 1)) / (8.0 * k);
            xp *= ax;
            const double t = a / xp, at = t < 0 ? -t : t;
            if (at > last || at < 1e-18) break;
            last = at;
            // even k -> P (sign (-1)^(k/2)), odd k -> Q (sign (-1)^((k-1)/2))
            const double sg = ((k / 2) % 2 == 0) ? 1.0 : -1.0;
            if (k % 2 == 0) p += sg * t;
            else q += sg * t;
        }
        const double w = ax - 0.75 * kPi;
        r = sqrt(2.0 / (kPi * ax)) * (p * cos(w) - q * sin(w));
    }
    return x < 0.0 ? -r : r;
}

// Power beam (2 J1(x) / x)^2 of Eq. airy at frequency nu and unit direction (east, north,
// up): x = (D_ns n^2 + D_ew e^2) / sqrt(e^2 + n^2) pi nu / c (the effective diameter
// D_ns + sin^2(az) (D_ew - D_ns) times sin(za)); zero at and below the horizon
__host__ __device__ inline double airy_power(double nu, double e, double n, double u, double dew, double dns)
{
    if (!(u > 0.0)) return 0.0;
    const double rho2 = e * e + n * n;
    if (rho2 == 0.0) return 1.0;
    const double x = (dns * n * n + dew * e * e) / sqrt(rho2) * kPi * nu / kCLight;
    if (x < 1e-4) {
        const double a = 1.0 - x * x / 8.0;
        return a * a;
    }
    const double a = 2.0 * bessel_j1(x) / x;
    return a * a;
}

template <typename R> struct Tab;
template <> struct Tab<double> {
    static __device__ __forceinline__ const double *domega(const DevGeom &g) { return g.domega64; }
    static __device__ __forceinline__ const double *za2(const DevGeom &g) { return g.za2_64; }
    static __device__ __forceinline__ const double *gleg(const DevGeom &g) { return g.gleg64; }
    static __device__ __forceinline__ const double *bcoef(const DevGeom &g) { return g.bcoef64; }
};
template <> struct Tab<float> {
    static __device__ __forceinline__ const float *domega(const DevGeom &g) { return g.domega32; }
    static __device__ __forceinline__ const float *za2(const DevGeom &g) { return g.za2_32; }
    static __device__ __forceinline__ const float *gleg(const DevGeom &g) { return g.gleg32; }
    static __device__ __forceinline__ const float *bcoef(const DevGeom &g) { return g.bcoef32; }
};

// Hour-angle form of the contraction for drift scans (k_ha.cu): valid when the LSTs are
// spaced by an integer number k of RA pixels, so that the direction of pixel (r, d) at
// LST t depends on n = t k - r + R - 1 only.
struct HaState {
    bool on = false;
    int k = 1;                 // LST step in hour-angle cells
    int q = 1;                 // hour-angle cells per RA pixel (the LST step is k / q pixels)
    int nh = 0, nhp = 0;       // hour-angle indices used, padded to a multiple of 128
    int nbc = 0;               // 64-index chunks per declination row (nhp / 64)
    int U = 0;                 // fringe groups: baselines with equal vectors up to sign
    int nant = 0;              // antennas in the phasor table (a subset covering every group)
    int ant_of[64] = {};       // table entry -> antenna
    int nmt = 0;               // forward M-tiles, ceil(U / 64)
    int nkq = 0;               // adjoint K-chunks, ceil(U / 32)
    int npad = 0;              // LSTs per pass (at most 64) rounded up to 16 (MMA N)
    int Jc = 0, Ly = 0;        // forward sky image chunks; sky-strip length (16-bit elements)
    int Lyc = 0;               // strip elements one pass of at most 64 LSTs reads
    int grid = 0, J = 0;       // forward CTAs; partial sums per (M-tile, channel) segment (vpart stride)
    int J_alloc = 0;           // J of the default grid (the allocation)
    int grid_adj = 0;          // adjoint CTAs (0: one per SM)
    float sp = 1.f;            // response scale 2^e (e even): the table holds sqrt(dOmega A) 2^(e/2)
    float2 *E = nullptr;       // [F][D][nbc][nant + 1][66] phasor table, cells paired (entry nant is zero; 2 pad cells)
    float2 *Ea = nullptr;      // the same table with one (Re, Im) per cell, for the adjoint
    int2 *uij = nullptr;       // [nmt * 64] representative pair (table entries) of each group; padding (nant, nant)
    int *bmap = nullptr;       // [B] group * 2 + (1 if the baseline is the reversed vector)
    int *moff = nullptr;       // [U + 1] CSR offsets of group members
    int *mem = nullptr;        // [B] members, b * 2 + reversed
    int *ncontrib = nullptr;   // [nmt * F] forward CTAs contributing to each segment
    uint16_t *ys = nullptr;    // [2][F][D][Ly] scaled sky strips in the forward's cell order, hi then lo
    unsigned *xmax = nullptr;  // [F] max |x| of the centred sky per channel, as float bits
    float *ug = nullptr;       // [F][T][U][2] monopole visibility of each group (k_ha_monopole)
    float *vpart = nullptr;    // [nmt * F][J][128][npad] forward partial sums
    float *q32 = nullptr;      // [F][T][U][2] residual weights summed per group
    float *qmax_ft = nullptr;  // [F][T] max |Re Q|, |Im Q| per (channel, LST)
    float *qscale = nullptr;   // [F]
    uint8_t *qimg = nullptr;   // [F][nkq][2][npad * 128] swizzled B tiles of the adjoint
    std::vector<int> rep_ant;  // [U][2] antennas of each group's representative pair (host)
    double lst0 = 0.0, dra = 0.0;
};

// Mode <-> pixel transforms on the tensor cores (k_modes.cu): FP16 hi/lo images of the
// basis tables, 128-byte-swizzled per 64-wide K atom.
struct ModesTc {
    bool on = false;
    uint8_t *leg_img = nullptr;    // Leg [D tiles of 128][N]   (forward, first product)
    uint8_t *phi_img = nullptr;    // Phi [R][M]                 (forward, second product)
    uint8_t *phit_img = nullptr;   // Phi^T [M tiles of 128][R]  (adjoint, first product)
    uint8_t *legt_img = nullptr;   // Leg^T [N][D]               (adjoint, second product)
};

// Device parameter block of the HMC chain (k_chain.cu), rewritten before every call.
struct ChainDev {
    double eps0, a_min;               // initial (and largest) step, acceptance threshold of the step rule
    uint32_t k0, k1;                  // Philox key: the seed
    double it0;                       // iteration number at the start of the call (trace index origin)
    double *trace;                    // [ntrace][5] per iteration: eps used, H0, H1, accepted, a (or NULL)
    long long ntrace;
};

// Device workspace and state of one handle.
struct Ctx {
    fm_config cfg;
    std::vector<double> ant, freq, lst;
    int A, F, T, R, D, M, N, NG, npix, nk, B, prec;
    int64_t n_sky, n_par, n_vis;     // parameter space: sky modes (K x nk or F x nk) + gains
    // Legendre-in-frequency compression (K > 0): the model runs on n_sky_m = F x nk expanded modes
    int K = 0;
    int64_t n_sky_m = 0;
    void *fx64 = nullptr, *fx32 = nullptr;   // X[f][k] = P_k(nu^_f)
    std::vector<double> fx_host;
    void *ax = nullptr, *avx = nullptr, *gx = nullptr;   // expanded theta, v and gradient sky parts
    double *pc_gacc = nullptr;               // preconditioner: one channel's blocks before spreading
    size_t pc_gacc_n = 0;                    // its length in doubles
    size_t rsz;                       // bytes per real (4 or 8)
    DevGeom g;
    // owned device buffers
    std::vector<void *> allocs;
    void *data = nullptr, *mu = nullptr, *lam = nullptr;
    bool have_data = false, have_prior = false;
    void *x = nullptr, *xv = nullptr, *xbar = nullptr, *tmp = nullptr;
    void *vis = nullptr, *dvis = nullptr, *omega = nullptr, *zpart = nullptr;
    void *gains = nullptr, *dgains = nullptr, *work_par = nullptr;
    double *chi2p = nullptr, *scal = nullptr, *red = nullptr;
    int *status = nullptr;
    unsigned *ticket = nullptr;   // last-CTA ticket of k_prior_total (0 between launches)
    // preconditioner
    int pc_block = 0;
    double *pc_blocks = nullptr;      // FP64 GN blocks (sky then gain)
    void *pc_chol = nullptr;          // factors in the working real type
    void *pc_ginv = nullptr;          // gain block (block 64 only), FP64: L_g, L_g^-1, L_g^-T and L_g^-T L_g^-1
    void *pc_linv = nullptr;          // inverses of the 64 x 64 sky-block factors (block 64 only)
    double *pc_tmp = nullptr;         // FP64 scratch of the gain-block inverse
    int64_t pc_size = 0;
    int *pc_grp = nullptr;            // baseline groups of the build: rep [U][2], CSR offsets [U + 1], members [B]
    int pc_U = 0;
    // tensor-core path: per-channel power-of-two operand scale (FP16 modes), max cell solid angle
    float *tc_scale = nullptr;
    float *tc_wbar = nullptr;         // [F][T][npix] beam-weighted pixel adjoint per LST
    float domega_max = 0.f;
    // monopole split (FP32 storage paths): U[f][t][b] = visibility of a unit uniform sky,
    // computed once in FP64; the contraction kernels see x - a_00 only
    bool dc_split = false;
    float *dc_u = nullptr;
    void *dc_mean = nullptr;          // [F] channel means for fm_forward_pixels
    // profiling: event pairs around the contraction kernels
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_rec;
    size_t prof_next = 0;
    HaState ha;
    ModesTc mtc;
    // leapfrog scratch
    void *lf_q0 = nullptr, *lf_g = nullptr, *lf_z = nullptr;
    void *lf_y = nullptr;             // [gain-block order] FP64 intermediate of the dense solves
    double *lf_scal = nullptr;
    double *lf_prm = nullptr;         // [2] eps, accept uniform of fm_leapfrog (read by the kernels)
    // HMC chain (fm_hmc_chain): momentum buffers, device parameter block, the captured iteration
    void *ch_z = nullptr, *ch_p = nullptr;
    ChainDev *ch_dev = nullptr;
    ChainDev ch_host{};
    double *ch_h = nullptr;           // [2] H0, H1 of the last trajectory
    int *ch_acc = nullptr;
    cudaGraph_t ch_graph = nullptr;
    cudaGraphExec_t ch_exec = nullptr;
    void *ch_q = nullptr;
    double *ch_state = nullptr;
    int ch_steps = 0;
    // delay filter along frequency (Eq. rime_filter): F [F][F] and the weights 1 / N~_ff in the
    // working type, the residual buffer and the chi^2 partials of the filter pass
    bool df_on = false;
    void *df_F = nullptr, *df_w = nullptr, *df_r = nullptr;
    double *df_chi2p = nullptr;
    int df_nparts = 0;
};

void chain_release(Ctx &c);           // the chain's graph (k_chain.cu)

// --------------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
fm_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define FM_CK(call)                                                         \
    do {                                                                    \
        cudaError_t _e = (call);                                            \
        if (_e != cudaSuccess) return ::fm::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

extern long long g_launches;     // kernels launched by the library (relaxed counter)
#define FM_CK_LAUNCH()                                                      \
    do {                                                                    \
        __atomic_fetch_add(&::fm::g_launches, 1LL, __ATOMIC_RELAXED);       \
        FM_CK(cudaGetLastError());                                          \
    } while (0)

// Lets kernel `fn` launch with up to the device's opt-in shared memory per block (less its
// static shared memory).  The limit
// is an attribute of the function, shared by every handle in the process, so it is raised to
// the device maximum instead of being set to one handle's size (a smaller size set for one
// handle would make another handle's launches, or graph nodes captured from them, fail).
template <typename F>
inline cudaError_t smem_opt_in(F fn)
{
    int dev = 0, mx = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);   // the kernel's static shared memory counts too
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
}

#define FM_TRY(expr)                                                        \
    do {                                                                    \
        fm_status _s = (expr);                                              \
        if (_s != FM_OK) return _s;                                         \
    } while (0)

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ profiling
inline cudaEvent_t prof_event(Ctx &c)
{
    if (c.prof_next >= c.prof_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c.prof_pool.push_back(e);
    }
    return c.prof_pool[c.prof_next++];
}

// records an event pair of class `cls` (0 forward contraction kernel, 1 adjoint
// contraction kernel) around the work `fn` enqueues on `st`
template <typename F>
fm_status profiled(Ctx &c, int cls, cudaStream_t st, F fn)
{
    if (!c.prof_on) return fn();
    cudaEvent_t a = prof_event(c), b = prof_event(c);
    if (!a || !b) return fn();
    cudaEventRecord(a, st);
    fm_status s = fn();
    cudaEventRecord(b, st);
    c.prof_rec.push_back({cls, {a, b}});
    return s;
}

// ------------------------------------------------------------ stage launchers
// (each defined in the .cu file that owns the kernels; all enqueue on `st`)
fm_status launch_precompute(Ctx &c, cudaStream_t st);

// Sky strips of the hour-angle forward written by the tensor-core mode transform: element
// j = off + r q of the strip of (channel f, declination d), at hi/lo + (f D + d) Ly + j, holds
// sc x[f][d][r] split into 16-bit hi / lo parts (FP16 or BF16), sc = 2^(14 - e) for the
// channel's largest |x| in [2^(e-1), 2^e); the other elements stay zero.
struct StripArgs {
    uint16_t *hi = nullptr, *lo = nullptr;
    int Ly = 0, off = 0, q = 1, bf16 = 0;
};
// the hour-angle form's strips as a StripArgs when the transform can write them (one CTA
// per channel: at most 128 declinations)
bool ha_strip_args(const Ctx &c, StripArgs &sa);

template <typename R>
// a -> x; xmax != NULL (tensor-core transform only): also each channel's largest |x| (as
// float bits) into xmax[f] (atomicMax into a zeroed xmax; with strips, a plain store and the
// strips of the hour-angle forward as well)
fm_status launch_modes_forward(Ctx &c, const R *a, R *x, cudaStream_t st, int skip_dc = 0, unsigned *xmax = nullptr,
                               const StripArgs *strips = nullptr);
template <typename R>
fm_status launch_modes_adjoint(Ctx &c, const R *xbar, R *abar, cudaStream_t st);  // xbar -> abar
template <typename R>
fm_status launch_gains(Ctx &c, const R *gamma, R *g, cudaStream_t st);       // theta gain part -> g[F][A]
template <typename R>
fm_status launch_vis(Ctx &c, const R *x, R *vis, cudaStream_t st);           // x -> V (unit gains)
template <typename R>
fm_status launch_adjoint(Ctx &c, const R *omega, R *xbar, cudaStream_t st);  // omega -> xbar
template <typename R>
fm_status launch_apply_gains(Ctx &c, const R *vis, const R *g, R *out, cudaStream_t st);
template <typename R>
fm_status launch_chi2_mid(Ctx &c, const R *vis, const R *g, R *omega, R *zpart, double *chi2p,
                          cudaStream_t st);
template <typename R>
fm_status launch_hvp_mid(Ctx &c, const R *vis, const R *dvis, const R *g, const R *dg, int full, R *omega,
                         R *zpart, cudaStream_t st);
template <typename R>
fm_status launch_gain_reduce(Ctx &c, const R *zpart, R *grad_gain, cudaStream_t st);
// per-(channel, LST) form of the chi^2 epilogue (gradient path): chi2p[f][t], the gain
// partials zpart[f][t][a][2], omega, or (groups) the hour-angle group sums of omega; the
// gains are formed inside from the coefficients gamma [A][NG][2]
// The hour-angle forward's unfinished output (one pass over the LSTs), from which the chi^2
// epilogue forms V itself: V_b = sc (S[2u], s S[2u+1]) + c_f (Ug_re[u], s Ug_im[u]) for member
// b of group u (s = -1 when reversed), S = the sum over the segment's contributors of the
// partial rows at the CTA's LST, sc = 1 / (sp 2^(14-e)) for the channel maximum xmax[f] in
// [2^(e-1), 2^e), c_f = dc[f dcs] (0 without the monopole split).
struct HaVSrc {
    const float *vpart = nullptr;    // [nmt F][J][npad][128]
    const int *ncontrib = nullptr;   // [nmt F]
    const int *bmap = nullptr;       // [B] 2 u + reversed
    const unsigned *xmax = nullptr;  // [F]
    const float *dc = nullptr;
    long long dcs = 0;
    const float *ug = nullptr;       // [F][T][U][2]
    float sp = 1.f;
    int J = 0, npad = 0, nmt = 0, F = 0;
};
// fills v when the epilogue can form V from the partials (hour-angle form on, one LST pass,
// the groups' monopole visibilities present when dc != nullptr)
bool ha_vsrc(const Ctx &c, const float *dc, long long dcs, HaVSrc &v);

template <typename R>
fm_status launch_chi2_chan(Ctx &c, const R *vis, const R *gamma, R *omega, R *zpart, double *chi2p, bool groups,
                           cudaStream_t st, const R *rin = nullptr, const HaVSrc *hv = nullptr);
// grad_gain from zpart in one pass over (channel, LST)
template <typename R>
fm_status launch_gain_reduce_chan(Ctx &c, const R *zpart, R *grad_gain, cudaStream_t st);
template <typename R>
// with kick_p != NULL also the momentum kick kick_p -= kick_frac eps grad, eps = kick_prm[0] (device)
fm_status launch_prior_and_total(Ctx &c, const R *theta, R *grad, const double *chi2p, int nchi2, double *chi2_out,
                                 double *u_out, cudaStream_t st, R *kick_p = nullptr,
                                 const double *kick_prm = nullptr, double kick_frac = 0.0);
template <typename R>
fm_status launch_prior_hvp(Ctx &c, const R *v, R *hv, cudaStream_t st);
template <typename R>
fm_status launch_add_dc(Ctx &c, const R *src, long long stride, R *vis, cudaStream_t st);
template <typename R>
fm_status launch_center(Ctx &c, const R *x, R *xc, R *mean, cudaStream_t st);
// visibilities of the sky of mode coefficients a (the sky part of theta): V = V(x - a_00) + a_00 U
// on the FP32 paths, V(x) directly on the FP64 path; x is left in `xbuf`
fm_status launch_d2f(long long n, const double *a, float *b, cudaStream_t st);
template <typename R>
fm_status vis_of_modes(Ctx &c, const R *a, R *xbuf, R *vis, cudaStream_t st, bool partials_only = false);

// tensor-core contraction (sm_103a tcgen05); returns FM_ERR_UNSUPPORTED when the
// shape does not fit its tiles
fm_status launch_vis_tc(Ctx &c, const float *x, float *vis, cudaStream_t st);
fm_status launch_adjoint_tc(Ctx &c, const float *omega, float *xbar, cudaStream_t st);
// hour-angle form (drift scans with the LST step a whole number of RA pixels); ha_setup
// leaves c.ha.on false when the geometry, precision or sizes do not allow it
fm_status ha_setup(Ctx &c);
// monopole visibilities U[f][t][b] = V_b(1) in FP64 through the hour-angle geometry
// (FM_ERR_UNSUPPORTED when the form is off or its tiles do not fit)
fm_status ha_monopole(Ctx &c, float *U, cudaStream_t st);
// launch grids of the hour-angle contraction kernels (0: one CTA per SM)
fm_status ha_set_grids(Ctx &c, int ctas_fwd, int ctas_adj);
// tensor-core mode transforms (float handles of the split precisions)
fm_status modes_tc_setup(Ctx &c);
fm_status launch_modes_tc_forward(Ctx &c, const float *a, float *x, cudaStream_t st, int skip_dc, unsigned *xmax,
                                  const StripArgs *strips = nullptr);
fm_status launch_modes_tc_adjoint(Ctx &c, const float *xbar, float *abar, cudaStream_t st);
fm_status launch_modes_tc_adjoint_maps(Ctx &c, const float *xbar, int nmaps, float *abar, cudaStream_t st);
// dc != nullptr: also adds the monopole visibilities dc[f * dcs] U[f][t][b]; xmax_ready: the
// channel maxima of x are already in c.ha.xmax (formed by the mode transform); strips_ready:
// so are the sky strips of x (written by the mode transform); partials_only: V is not
// finished (the forward's partial sums stay in c.ha.vpart for the chi^2 epilogue, HaVSrc)
fm_status launch_vis_ha(Ctx &c, const float *x, float *vis, cudaStream_t st, const float *dc = nullptr,
                        long long dcs = 0, bool xmax_ready = false, bool strips_ready = false,
                        bool partials_only = false);
// q_ready: the group sums q32 / qmax_ft were already formed from omega (by the chi^2 epilogue)
fm_status launch_adjoint_ha(Ctx &c, const float *omega, float *xbar, cudaStream_t st, bool q_ready = false);

// delay filter (k_filter.cu): r = g_p conj(g_q) V - d into c.df_r, then in place
// r <- sigma^2 F^T W F r with the filtered chi^2 partials in c.df_chi2p
template <typename R>
fm_status launch_delay_filter(Ctx &c, const R *vis, const R *gamma, cudaStream_t st);

// Legendre-in-frequency compression (k_freq.cu): a[f][j] = sum_k X_k(nu_f) a~[k][j] and its
// transpose; the preconditioner spreads a channel's FP64 blocks G into the K compressed ones
fm_status freq_basis_setup(Ctx &c);
template <typename R>
fm_status launch_freq_expand(Ctx &c, const R *ap, R *am, cudaStream_t st);
template <typename R>
fm_status launch_freq_contract(Ctx &c, const R *gm, R *gp, cudaStream_t st);
fm_status launch_freq_spread(Ctx &c, int f, long long n, const double *G, double *acc, cudaStream_t st);

// preconditioner and leapfrog
template <typename R>
fm_status run_build_precond(Ctx &c, const R *theta, int block, cudaStream_t st);
template <typename R>
fm_status run_precond_apply(Ctx &c, int op, const R *in, R *out, cudaStream_t st);
template <typename R>
fm_status set_leapfrog_params(Ctx &c, double eps, double u, cudaStream_t st);
template <typename R>
fm_status prepare_leapfrog(Ctx &c);
template <typename R>
fm_status run_leapfrog(Ctx &c, R *q, R *p, const double *prm, int n_steps, double *h_out, int *acc_out,
                       cudaStream_t st);

// gradient / hvp drivers (fm_api.cu)
// with kick_p != NULL the evaluation ends with the leapfrog kick kick_p -= kick_frac eps grad,
// eps = kick_prm[0] (device), fused into its last pass over the gradient
template <typename R>
fm_status run_chi2_grad(Ctx &c, const R *theta, double *chi2_out, double *u_out, R *grad, cudaStream_t st,
                        R *kick_p = nullptr, const double *kick_prm = nullptr, double kick_frac = 0.0);

}  // namespace fm
