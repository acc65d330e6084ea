// Delay filter along frequency (Eq. rime_filter, Eq. gpr, Eq. filtered_noise).
//
// The model and the data are both filtered, m = F y', with the Gaussian-process high-pass
// filter F = I - C_fg (C_fg + C_noise)^-1 of Eq. gpr: C_fg[k][l] = sinc(2 tau_max (nu_k - nu_l))
// (a top-hat of half-width tau_max in delay) and C_noise = noise_ratio C_fg(0) I.  F is real and
// acts on every (LST, baseline) column of the visibilities along frequency.  The likelihood
// keeps a diagonal noise, N~_ff = sigma^2 sum_g F_fg^2 (the diagonal of F N F^T,
// Eq. filtered_noise), so
//   chi^2 = sum_{f, t, b} |r~_ftb|^2 / N~_ff,  r~ = F (m - d)  (per column),
// and the residual weights of the adjoint become F^T (r~ / N~): the chi^2 epilogue then runs
// on sigma^2 F^T (r~ / N~) in place of m - d.  F is built once on the host in FP64 (a
// Cholesky factorisation of C_fg + C_noise), then applied in the working type.
#include <cmath>
#include <vector>

#include "fm_internal.cuh"

namespace fm {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

constexpr int DF_COLS = 32;       // (LST, baseline) columns per CTA
constexpr int DF_THREADS = 256;

// r[f][t][b] = g_i(f) conj(g_j(f)) V - d: one CTA per (channel, LST), gains formed in shared
// memory from the coefficients as the chi^2 epilogue forms them
template <typename R>
__global__ void __launch_bounds__(256) k_df_resid(DevGeom g, const R *__restrict__ vis, const R *__restrict__ data,
                                                  const R *__restrict__ gamma, R *__restrict__ r)
{
    using C2 = typename Cx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sG = reinterpret_cast<C2 *>(smem_raw);
    const int ft = blockIdx.x, f = ft / g.T;
    const R *X = Tab<R>::gleg(g) + (size_t)f * g.NG;
    for (int i = threadIdx.x; i < g.A; i += blockDim.x) {
        R re = 0, im = 0;
        for (int k = 0; k < g.NG; ++k) {
            re += X[k] * gamma[(i * g.NG + k) * 2];
            im += X[k] * gamma[(i * g.NG + k) * 2 + 1];
        }
        sG[i].x = re;
        sG[i].y = im;
    }
    __syncthreads();
    const C2 *vrow = reinterpret_cast<const C2 *>(vis) + (size_t)ft * g.B;
    const C2 *drow = reinterpret_cast<const C2 *>(data) + (size_t)ft * g.B;
    C2 *rrow = reinterpret_cast<C2 *>(r) + (size_t)ft * g.B;
    for (int b = threadIdx.x; b < g.B; b += blockDim.x) {
        const C2 V = vrow[b], d = drow[b], gi = sG[g.bl_i[b]], gj = sG[g.bl_j[b]];
        const R ggr = gi.x * gj.x + gi.y * gj.y, ggi = gi.y * gj.x - gi.x * gj.y;
        C2 o;
        o.x = ggr * V.x - ggi * V.y - d.x;
        o.y = ggr * V.y + ggi * V.x - d.y;
        rrow[b] = o;
    }
}

// In place, per column q = t B + b of r[f][q]: r~ = F r, the CTA's chi^2 partial
// sum_f w_f |r~_f|^2 (FP64 across warps), then r <- sigma^2 F^T (w r~).  A warp holds one
// channel row at a time (F read as a broadcast), its lanes the CTA's 32 columns.
template <typename R>
__global__ void __launch_bounds__(DF_THREADS) k_df_apply(int nf, long long ncol, R sigma2, const R *__restrict__ Fm,
                                                         const R *__restrict__ w, R *__restrict__ r,
                                                         double *__restrict__ chi2p)
{
    using C2 = typename Cx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sF = reinterpret_cast<R *>(smem_raw);                       // [nf][nf]
    C2 *sA = reinterpret_cast<C2 *>(sF + (size_t)nf * nf + (nf & 1));   // [nf][DF_COLS]
    C2 *sB = sA + (size_t)nf * DF_COLS;                            // [nf][DF_COLS]
    __shared__ double red[DF_THREADS / 32];
    const int tid = threadIdx.x, c = tid & 31, w0 = tid >> 5;
    const long long q0 = (long long)blockIdx.x * DF_COLS;
    const long long q = q0 + c;
    C2 *rc = reinterpret_cast<C2 *>(r);
    for (int e = tid; e < nf * nf; e += DF_THREADS) sF[e] = Fm[e];
    for (int f = w0; f < nf; f += DF_THREADS / 32) {
        C2 v;
        v.x = v.y = R(0);
        if (q < ncol) v = rc[(size_t)f * ncol + q];
        sA[f * DF_COLS + c] = v;
    }
    __syncthreads();
    R c2 = 0;
    for (int f = w0; f < nf; f += DF_THREADS / 32) {
        R ar = 0, ai = 0;
        for (int g2 = 0; g2 < nf; ++g2) {
            const R fv = sF[f * nf + g2];
            const C2 v = sA[g2 * DF_COLS + c];
            ar += fv * v.x;
            ai += fv * v.y;
        }
        const R wf = w[f];
        c2 += wf * (ar * ar + ai * ai);
        C2 s;
        s.x = wf * ar;
        s.y = wf * ai;
        sB[f * DF_COLS + c] = s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    if (c == 0) red[w0] = (double)c2;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < DF_THREADS / 32; ++k) a += red[k];
        chi2p[blockIdx.x] = a;
    }
    for (int f = w0; f < nf; f += DF_THREADS / 32) {
        R ar = 0, ai = 0;
        for (int g2 = 0; g2 < nf; ++g2) {
            const R fv = sF[g2 * nf + f];
            const C2 v = sB[g2 * DF_COLS + c];
            ar += fv * v.x;
            ai += fv * v.y;
        }
        if (q < ncol) {
            C2 o;
            o.x = sigma2 * ar;
            o.y = sigma2 * ai;
            rc[(size_t)f * ncol + q] = o;
        }
    }
}

template <typename R>
size_t df_smem(int nf)
{
    return sizeof(R) * ((size_t)nf * nf + (nf & 1)) + 2 * sizeof(typename Cx<R>::t) * (size_t)nf * DF_COLS;
}

// F = I - C (C + eps I)^-1 in FP64: Cholesky of M = C + eps I, Y = M^-1 C column by column,
// F = I - Y^T (C and M^-1 are symmetric).  Returns false if M is not positive definite.
bool build_filter(const std::vector<double> &nu, double tau, double eps, std::vector<double> &F)
{
    const int n = (int)nu.size();
    std::vector<double> C((size_t)n * n), L((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
            const double x = 2.0 * tau * (nu[k] - nu[l]);
            C[(size_t)k * n + l] = x == 0.0 ? 1.0 : std::sin(kPi * x) / (kPi * x);
        }
    for (int k = 0; k < n; ++k)
        for (int l = 0; l <= k; ++l) {
            double a = C[(size_t)k * n + l] + (k == l ? eps : 0.0);
            for (int m = 0; m < l; ++m) a -= L[(size_t)k * n + m] * L[(size_t)l * n + m];
            if (k == l) {
                if (!(a > 0.0)) return false;
                L[(size_t)k * n + k] = std::sqrt(a);
            } else {
                L[(size_t)k * n + l] = a / L[(size_t)l * n + l];
            }
        }
    F.assign((size_t)n * n, 0.0);
    std::vector<double> y(n);
    for (int col = 0; col < n; ++col) {
        for (int k = 0; k < n; ++k) {              // L z = C[:, col]
            double a = C[(size_t)k * n + col];
            for (int m = 0; m < k; ++m) a -= L[(size_t)k * n + m] * y[m];
            y[k] = a / L[(size_t)k * n + k];
        }
        for (int k = n - 1; k >= 0; --k) {         // L^T y = z
            double a = y[k];
            for (int m = k + 1; m < n; ++m) a -= L[(size_t)m * n + k] * y[m];
            y[k] = a / L[(size_t)k * n + k];
        }
        for (int k = 0; k < n; ++k) F[(size_t)col * n + k] = (col == k ? 1.0 : 0.0) - y[k];   // row col of I - Y^T
    }
    return true;
}

template <typename R>
fm_status upload_filter(Ctx &c, const std::vector<double> &F, const std::vector<double> &w)
{
    const size_t nf = (size_t)c.F;
    if (!c.df_F) {
        const long long ncol = (long long)c.T * c.B;
        c.df_nparts = (int)cdiv(ncol, DF_COLS);
        if (cudaMalloc(&c.df_F, sizeof(R) * nf * nf) != cudaSuccess ||
            cudaMalloc(&c.df_w, sizeof(R) * nf) != cudaSuccess ||
            cudaMalloc(&c.df_r, sizeof(R) * 2 * (size_t)c.n_vis) != cudaSuccess ||
            cudaMalloc(&c.df_chi2p, sizeof(double) * (size_t)c.df_nparts) != cudaSuccess) {
            set_error("cudaMalloc delay filter");
            return FM_ERR_ALLOC;
        }
        c.allocs.push_back(c.df_F);
        c.allocs.push_back(c.df_w);
        c.allocs.push_back(c.df_r);
        c.allocs.push_back(c.df_chi2p);
    }
    std::vector<R> fr(F.begin(), F.end()), wr(w.begin(), w.end());
    FM_CK(cudaMemcpy(c.df_F, fr.data(), sizeof(R) * fr.size(), cudaMemcpyHostToDevice));
    FM_CK(cudaMemcpy(c.df_w, wr.data(), sizeof(R) * wr.size(), cudaMemcpyHostToDevice));
    return FM_OK;
}

}  // namespace

template <typename R>
fm_status launch_delay_filter(Ctx &c, const R *vis, const R *gamma, cudaStream_t st)
{
    k_df_resid<R><<<c.F * c.T, 256, sizeof(typename Cx<R>::t) * (size_t)c.A, st>>>(c.g, vis, (const R *)c.data, gamma,
                                                                              (R *)c.df_r);
    FM_CK_LAUNCH();
    const long long ncol = (long long)c.T * c.B;
    const size_t smem = df_smem<R>(c.F);
    FM_CK(smem_opt_in(k_df_apply<R>));
    k_df_apply<R><<<(unsigned)c.df_nparts, DF_THREADS, smem, st>>>(c.F, ncol, (R)(1.0 / c.g.inv_sigma2),
                                                                  (const R *)c.df_F, (const R *)c.df_w, (R *)c.df_r,
                                                                  c.df_chi2p);
    FM_CK_LAUNCH();
    return FM_OK;
}
template fm_status launch_delay_filter<float>(Ctx &, const float *, const float *, cudaStream_t);
template fm_status launch_delay_filter<double>(Ctx &, const double *, const double *, cudaStream_t);

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_set_delay_filter(fm_handle h, double tau_max_s, double noise_ratio)
{
    if (!h) {
        set_error("invalid argument: handle is NULL");
        return FM_ERR_INVALID_ARG;
    }
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (!(tau_max_s > 0.0)) {          // 0 (or less) switches the filter off
        c.df_on = false;
        return FM_OK;
    }
    if (!std::isfinite(tau_max_s) || !(noise_ratio > 0.0) || !std::isfinite(noise_ratio)) {
        set_error("invalid argument: tau_max_s must be finite and noise_ratio > 0");
        return FM_ERR_INVALID_ARG;
    }
    const bool fp64 = c.prec == FM_PREC_FP64_SIMT;
    if (df_smem<float>(c.F) * (fp64 ? 2 : 1) > 200 * 1024) {
        set_error("delay filter: %d channels exceed the filter kernel's shared memory", c.F);
        return FM_ERR_UNSUPPORTED;
    }
    std::vector<double> F;
    if (!build_filter(c.freq, tau_max_s, noise_ratio, F)) {
        set_error("delay filter: C_fg + C_noise is not positive definite");
        return FM_ERR_INVALID_ARG;
    }
    const double s2 = 1.0 / c.g.inv_sigma2;
    std::vector<double> w(c.F);
    for (int f = 0; f < c.F; ++f) {
        double a = 0.0;
        for (int g2 = 0; g2 < c.F; ++g2) a += F[(size_t)f * c.F + g2] * F[(size_t)f * c.F + g2];
        w[f] = 1.0 / (s2 * a);
    }
    const fm_status s = fp64 ? upload_filter<double>(c, F, w) : upload_filter<float>(c, F, w);
    if (s != FM_OK) return s;
    c.df_on = true;
    return FM_OK;
}
