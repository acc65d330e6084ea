// Once-per-handle precompute on the device, in FP64 ("cached mode" of App. C):
// topocentric directions of every pixel at every LST, squared zenith angles for the
// beam, exact cell solid angles, the separable mode basis, the gain frequency basis,
// per-channel antenna phase slopes and the beam exponent per channel.  The FP32
// copies used by the fast paths are split into (hi, lo) pairs where the phase needs
// more than 24 bits.
#include "fm_internal.cuh"

namespace fm {
namespace {

__device__ __forceinline__ void split2(double v, float *out)
{
    float hi = __double2float_rn(v);
    out[0] = hi;
    out[1] = __double2float_rn(v - (double)hi);
}

struct PreArgs {
    int T, R, D, M, N, NG, F, A;
    double ra_min, ra_max, dec_min, dec_max, lat, fwhm, ref_hz;
    double fmin, fmax;
    const double *lst, *freq, *ant;
};

// Pixel (dec d, ra r) at LST t: hour angle H = LST - RA; east/north/up components of
// the unit vector at latitude lat (standard equatorial-to-horizon rotation).
__global__ void k_topocentric(PreArgs a, double *s64, float *s32, double *za2_64, float *za2_32)
{
    long long n = (long long)a.T * a.D * a.R;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % a.R);
        int d = (int)((e / a.R) % a.D);
        int t = (int)(e / ((long long)a.R * a.D));
        double dra = (a.ra_max - a.ra_min) / a.R, ddec = (a.dec_max - a.dec_min) / a.D;
        double ra = a.ra_min + (r + 0.5) * dra;
        double dec = a.dec_min + (d + 0.5) * ddec;
        double H = a.lst[t] - ra;
        double sd, cd, sh, ch, sl, cl;
        sincos(dec, &sd, &cd);
        sincos(H, &sh, &ch);
        sincos(a.lat, &sl, &cl);
        double sE = -cd * sh;
        double sN = cl * sd - sl * cd * ch;
        double sU = sl * sd + cl * cd * ch;
        s64[3 * e + 0] = sE;
        s64[3 * e + 1] = sN;
        s64[3 * e + 2] = sU;
        split2(sE, s32 + 6 * e + 0);
        split2(sN, s32 + 6 * e + 2);
        split2(sU, s32 + 6 * e + 4);
        double z2 = -1.0;
        if (sU > 0.0) {
            double za = acos(sU > 1.0 ? 1.0 : sU);
            z2 = za * za;
        }
        za2_64[e] = z2;
        za2_32[e] = (float)z2;
    }
}

__device__ void legendre_row(double x, int n, double *out, int stride)
{
    if (n <= 0) return;
    double p0 = 1.0;
    out[0] = p0;
    if (n == 1) return;
    double p1 = x;
    out[stride] = p1;
    for (int k = 1; k + 1 < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - (double)k * p0) / (k + 1.0);
        out[(size_t)(k + 1) * stride] = p2;
        p0 = p1;
        p1 = p2;
    }
}

__global__ void k_tables(PreArgs a, double *domega64, float *domega32, double *phi64, float *phi32,
                         double *leg64, float *leg32, double *gleg64, float *gleg32, double *kap64,
                         float *kap32, double *bcoef64, float *bcoef32)
{
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    int nthr = gridDim.x * blockDim.x;
    double dra = (a.ra_max - a.ra_min) / a.R, ddec = (a.dec_max - a.dec_min) / a.D;
    for (int d = tid; d < a.D; d += nthr) {
        double lo = a.dec_min + d * ddec, hi = a.dec_min + (d + 1) * ddec;
        double w = dra * (sin(hi) - sin(lo));
        domega64[d] = w;
        domega32[d] = (float)w;
        double dhat = 2.0 * ((a.dec_min + (d + 0.5) * ddec) - a.dec_min) / (a.dec_max - a.dec_min) - 1.0;
        legendre_row(dhat, a.N, leg64 + (size_t)d * a.N, 1);
        for (int n = 0; n < a.N; ++n) leg32[(size_t)d * a.N + n] = (float)leg64[(size_t)d * a.N + n];
    }
    for (long long e = tid; e < (long long)a.R * a.M; e += nthr) {
        int r = (int)(e / a.M), m = (int)(e % a.M);
        double ahat = 2.0 * kPi * ((a.ra_min + (r + 0.5) * dra) - a.ra_min) / (a.ra_max - a.ra_min);
        double v;
        if (m == 0) v = 1.0;
        else if (m == a.M - 1 && a.M >= 2) v = cos(0.5 * a.M * ahat);
        else {
            int k = (m + 1) / 2;
            v = (m % 2 == 1) ? cos(k * ahat) : sin(k * ahat);
        }
        phi64[e] = v;
        phi32[e] = (float)v;
    }
    for (int f = tid; f < a.F; f += nthr) {
        double nu = a.freq[f];
        double nhat = (a.fmax > a.fmin) ? 2.0 * (nu - a.fmin) / (a.fmax - a.fmin) - 1.0 : 0.0;
        legendre_row(nhat, a.NG, gleg64 + (size_t)f * a.NG, 1);
        for (int k = 0; k < a.NG; ++k) gleg32[(size_t)f * a.NG + k] = (float)gleg64[(size_t)f * a.NG + k];
        // Gaussian beam exp(-za^2 / (2 s^2)), s = FWHM(nu) / sqrt(8 ln 2), FWHM = fwhm * ref / nu
        double c = 0.0;
        if (a.fwhm > 0.0) {
            double fw = a.fwhm * a.ref_hz / nu;
            double sig = fw / sqrt(8.0 * log(2.0));
            c = -1.0 / (2.0 * sig * sig);
        }
        bcoef64[f] = c;
        bcoef32[f] = (float)c;
        for (int i = 0; i < a.A; ++i)
            for (int k = 0; k < 3; ++k) {
                double kv = nu * a.ant[3 * i + k] / kCLight;
                kap64[((size_t)f * a.A + i) * 3 + k] = kv;
                split2(kv, kap32 + ((size_t)f * a.A + i) * 6 + 2 * k);
            }
    }
}

__global__ void k_dompix(int npix, int R, const float *__restrict__ domega32, float *__restrict__ dompix)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) dompix[p] = domega32[p / R];
}

// power beam of Eq. airy per (channel, LST, pixel), FP64, stored in both types
__global__ void k_beam_airy(int F, long long tp, const double *__restrict__ freq, const double *__restrict__ s64,
                            double dew, double dns, float *__restrict__ b32, double *__restrict__ b64)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)F * tp;
         e += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(e / tp);
        const double *s = s64 + 3 * (e % tp);
        const double v = airy_power(freq[f], s[0], s[1], s[2], dew, dns);
        b32[e] = (float)v;
        if (b64) b64[e] = v;
    }
}

}  // namespace

fm_status launch_precompute(Ctx &c, cudaStream_t st)
{
    PreArgs a;
    a.T = c.T; a.R = c.R; a.D = c.D; a.M = c.M; a.N = c.N; a.NG = c.NG; a.F = c.F; a.A = c.A;
    a.ra_min = c.cfg.ra_min; a.ra_max = c.cfg.ra_max; a.dec_min = c.cfg.dec_min; a.dec_max = c.cfg.dec_max;
    a.lat = c.cfg.latitude_rad; a.fwhm = c.cfg.beam_fwhm_ref_rad; a.ref_hz = c.cfg.beam_ref_hz;
    a.fmin = c.freq[0]; a.fmax = c.freq[0];
    for (double f : c.freq) { if (f < a.fmin) a.fmin = f; if (f > a.fmax) a.fmax = f; }
    // small host arrays go through a scratch device buffer owned by the handle
    size_t nbytes = sizeof(double) * (c.T + c.F + 3 * (size_t)c.A);
    double *tmp = nullptr;
    FM_CK(cudaMalloc(&tmp, nbytes));
    c.allocs.push_back(tmp);
    FM_CK(cudaMemcpyAsync(tmp, c.lst.data(), sizeof(double) * c.T, cudaMemcpyHostToDevice, st));
    FM_CK(cudaMemcpyAsync(tmp + c.T, c.freq.data(), sizeof(double) * c.F, cudaMemcpyHostToDevice, st));
    FM_CK(cudaMemcpyAsync(tmp + c.T + c.F, c.ant.data(), sizeof(double) * 3 * c.A, cudaMemcpyHostToDevice, st));
    a.lst = tmp; a.freq = tmp + c.T; a.ant = tmp + c.T + c.F;
    k_topocentric<<<1024, 256, 0, st>>>(a, const_cast<double *>(c.g.s64), const_cast<float *>(c.g.s32),
                                        const_cast<double *>(c.g.za2_64), const_cast<float *>(c.g.za2_32));
    FM_CK_LAUNCH();
    k_tables<<<64, 256, 0, st>>>(a, const_cast<double *>(c.g.domega64), const_cast<float *>(c.g.domega32),
                                 const_cast<double *>(c.g.phi64), const_cast<float *>(c.g.phi32),
                                 const_cast<double *>(c.g.leg64), const_cast<float *>(c.g.leg32),
                                 const_cast<double *>(c.g.gleg64), const_cast<float *>(c.g.gleg32),
                                 const_cast<double *>(c.g.kap64), const_cast<float *>(c.g.kap32),
                                 const_cast<double *>(c.g.bcoef64), const_cast<float *>(c.g.bcoef32));
    FM_CK_LAUNCH();
    k_dompix<<<cdiv(c.npix, 256), 256, 0, st>>>(c.npix, c.R, c.g.domega32, const_cast<float *>(c.g.dompix32));
    FM_CK_LAUNCH();
    c.g.freq64 = a.freq;
    if (c.g.beam32) {
        const long long tp = (long long)c.T * c.npix;
        k_beam_airy<<<2048, 256, 0, st>>>(c.F, tp, a.freq, c.g.s64, c.g.dish_ew, c.g.dish_ns,
                                          const_cast<float *>(c.g.beam32), const_cast<double *>(c.g.beam64));
        FM_CK_LAUNCH();
    }
    return FM_OK;
}

}  // namespace fm
