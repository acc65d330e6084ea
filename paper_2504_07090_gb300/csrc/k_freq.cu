// Legendre-in-frequency compression of the sky modes (Eq. fg_legendre, Eq. eor_model):
// a[f][j] = sum_{k < K} X_k(nu_f) a~[k][j], with X_k the Legendre polynomial P_k of the
// normalised frequency nu^ = 2 (nu - nu_min) / (nu_max - nu_min) - 1.  The parameters are then
// a~ (K x n_modes) and the gains; the model kernels run on the expanded per-channel modes, and
// gradients and Hessian-vector products come back through the transpose,
// g~[k][j] = sum_f X_k(nu_f) g[f][j].
#include <vector>

#include "fm_internal.cuh"

namespace fm {
namespace {

template <typename R>
__global__ void k_freq_expand(int F, int K, long long nk, const R *__restrict__ X, const R *__restrict__ ap,
                              R *__restrict__ am)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)F * nk;
         e += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(e / nk);
        const long long j = e % nk;
        R a = 0;
        for (int k = 0; k < K; ++k) a += X[(size_t)f * K + k] * ap[(size_t)k * nk + j];
        am[e] = a;
    }
}

template <typename R>
__global__ void k_freq_contract(int F, int K, long long nk, const R *__restrict__ X, const R *__restrict__ gm,
                                R *__restrict__ gp)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)K * nk;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / nk);
        const long long j = e % nk;
        R a = 0;
        for (int f = 0; f < F; ++f) a += X[(size_t)f * K + k] * gm[(size_t)f * nk + j];
        gp[e] = a;
    }
}

// acc[k][e] += X_k(nu_f)^2 G[e] for k < K: a channel's Gauss-Newton blocks into the blocks of
// the compressed parameters (the diagonal blocks in k of sum_f X_fk X_fk' H_f)
__global__ void k_freq_spread(long long n, int K, const double *__restrict__ Xf, const double *__restrict__ G,
                              double *__restrict__ acc)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double v = G[e];
        for (int k = 0; k < K; ++k) acc[(size_t)k * n + e] += Xf[k] * Xf[k] * v;
    }
}

}  // namespace

// X[f][k] = P_k(nu^_f) in FP64 (Bonnet's recursion) and FP32, uploaded once
fm_status freq_basis_setup(Ctx &c)
{
    if (c.K <= 0) return FM_OK;
    double fmin = c.freq[0], fmax = c.freq[0];
    for (double f : c.freq) {
        if (f < fmin) fmin = f;
        if (f > fmax) fmax = f;
    }
    std::vector<double> X((size_t)c.F * c.K);
    for (int f = 0; f < c.F; ++f) {
        const double x = fmax > fmin ? 2.0 * (c.freq[f] - fmin) / (fmax - fmin) - 1.0 : 0.0;
        double p0 = 1.0, p1 = x;
        for (int k = 0; k < c.K; ++k) {
            double v;
            if (k == 0) v = 1.0;
            else if (k == 1) v = x;
            else {
                v = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = v;
            }
            X[(size_t)f * c.K + k] = v;
        }
    }
    std::vector<float> X32(X.begin(), X.end());
    FM_CK(cudaMalloc(&c.fx64, sizeof(double) * X.size()));
    c.allocs.push_back(c.fx64);
    FM_CK(cudaMalloc(&c.fx32, sizeof(float) * X.size()));
    c.allocs.push_back(c.fx32);
    FM_CK(cudaMemcpy(c.fx64, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice));
    FM_CK(cudaMemcpy(c.fx32, X32.data(), sizeof(float) * X32.size(), cudaMemcpyHostToDevice));
    c.fx_host = X;
    const size_t n = (size_t)c.n_sky_m * c.rsz;
    for (void **p : {&c.ax, &c.avx, &c.gx}) {
        FM_CK(cudaMalloc(p, n));
        c.allocs.push_back(*p);
    }
    return FM_OK;
}

template <typename R>
fm_status launch_freq_expand(Ctx &c, const R *ap, R *am, cudaStream_t st)
{
    const R *X = std::is_same<R, float>::value ? (const R *)c.fx32 : (const R *)c.fx64;
    k_freq_expand<R><<<2048, 256, 0, st>>>(c.F, c.K, c.nk, X, ap, am);
    FM_CK_LAUNCH();
    return FM_OK;
}

template <typename R>
fm_status launch_freq_contract(Ctx &c, const R *gm, R *gp, cudaStream_t st)
{
    const R *X = std::is_same<R, float>::value ? (const R *)c.fx32 : (const R *)c.fx64;
    k_freq_contract<R><<<2048, 256, 0, st>>>(c.F, c.K, c.nk, X, gm, gp);
    FM_CK_LAUNCH();
    return FM_OK;
}

fm_status launch_freq_spread(Ctx &c, int f, long long n, const double *G, double *acc, cudaStream_t st)
{
    k_freq_spread<<<1024, 256, 0, st>>>(n, c.K, (const double *)c.fx64 + (size_t)f * c.K, G, acc);
    FM_CK_LAUNCH();
    return FM_OK;
}

template fm_status launch_freq_expand<float>(Ctx &, const float *, float *, cudaStream_t);
template fm_status launch_freq_expand<double>(Ctx &, const double *, double *, cudaStream_t);
template fm_status launch_freq_contract<float>(Ctx &, const float *, float *, cudaStream_t);
template fm_status launch_freq_contract<double>(Ctx &, const double *, double *, cudaStream_t);

}  // namespace fm
