// Hessian-preconditioned HMC pieces (Sec. 4.2 and App. B):
//   - the Gauss-Newton Hessian of U on a block diagonal, accumulated in FP64:
//       sky blocks from the response columns R_k(t, pq) = g_p conj(g_q) sum_pix phi_k
//       dOmega A K_pq, built per (channel, LST) through the separable basis (contract
//       RA, then Dec) and reduced into per-block Grams; the gain block from the
//       per-baseline sums S_pq(nu) = sum_t |V_pq|^2 (the only data it needs);
//   - Cholesky of every block with prior inflation until positive definite;
//   - leapfrog kicks, the drift q += eps L^-T L^-1 p, kinetic energy z.z/2 (L z = p)
//     in FP64, and the Metropolis test u < exp(H0 - H1) on the device.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fm_internal.cuh"
#include "tc_ptx.cuh"

namespace fm {

template <typename R> struct V2h;
template <> struct V2h<float> { using t = float2; };
template <> struct V2h<double> { using t = double2; };

__device__ __forceinline__ float phase_frac_2f_h(const float *__restrict__ kap, const float *__restrict__ s)
{
    float accf = 0.f, acce = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float kh = kap[2 * c], kl = kap[2 * c + 1], sh = s[2 * c], sl = s[2 * c + 1];
        float p = __fmul_rn(kh, sh);
        float e = __fmaf_rn(kh, sh, -p);
        float f = __fsub_rn(p, rintf(p));
        accf = __fadd_rn(accf, f);
        acce = __fadd_rn(acce, __fadd_rn(e, __fmaf_rn(kh, sl, __fmul_rn(kl, sh))));
    }
    float t = __fadd_rn(accf, acce);
    return __fsub_rn(t, rintf(t));
}

// Baseline fringe K_pq = E_p conj(E_q) at one pixel, from the two antenna phases.
__device__ __forceinline__ void fringe(const DevGeom &g, int f, int i, int j, int t, int p, float &kr, float &ki)
{
    const float *s = g.s32 + ((size_t)t * g.npix + p) * 6;
    float a = phase_frac_2f_h(g.kap32 + ((size_t)f * g.A + i) * 6, s);
    float b = phase_frac_2f_h(g.kap32 + ((size_t)f * g.A + j) * 6, s);
    float d = a - b;                                   // |d| <= 1: phase of b_pq . s nu / c in turns
    d -= rintf(d);
    float sn, cs;
    sincospif(2.f * d, &sn, &cs);
    kr = cs;
    ki = -sn;
}
__device__ __forceinline__ void fringe(const DevGeom &g, int f, int i, int j, int t, int p, double &kr, double &ki)
{
    const double *ki_ = g.kap64 + ((size_t)f * g.A + i) * 3, *kj = g.kap64 + ((size_t)f * g.A + j) * 3;
    const double *s = g.s64 + ((size_t)t * g.npix + p) * 3;
    double ph = (ki_[0] - kj[0]) * s[0] + (ki_[1] - kj[1]) * s[1] + (ki_[2] - kj[2]) * s[2];
    ph -= rint(ph);
    double sn, cs;
    sincospi(2.0 * ph, &sn, &cs);
    kr = cs;
    ki = -sn;
}

// Baselines with equal vectors b = r_p - r_q (to 1 nm) up to sign have the same fringe, or
// its conjugate, at every pixel (Eq. rime_discrete with one beam for all antennas), so their
// response columns R_k(t, pq) = g_p conj(g_q) S_k differ only by the gain factor and, for
// reversed vectors, a conjugation; the Gauss-Newton Gram Re(R_k^H R_k') / sigma^2 of a group
// is then W_u Re(conj(S_u,k) S_u,k') / sigma^2 with W_u = sum over members |g_p g_q|^2: one
// response per group.  pc_groups lists the groups (representative pair, CSR members).
static void pc_groups(const Ctx &c, std::vector<int> &rep, std::vector<int> &off, std::vector<int> &mem)
{
    std::vector<double> rb;
    std::vector<std::vector<int>> members;
    for (int i = 0, b = 0; i < c.A; ++i)
        for (int j = i + 1; j < c.A; ++j, ++b) {
            const double v0 = c.ant[3 * i] - c.ant[3 * j], v1 = c.ant[3 * i + 1] - c.ant[3 * j + 1],
                         v2 = c.ant[3 * i + 2] - c.ant[3 * j + 2];
            int found = -1;
            for (size_t u = 0; u < members.size() && found < 0; ++u) {
                const double *r = &rb[3 * u];
                const double dp = std::fmax(std::fabs(v0 - r[0]), std::fmax(std::fabs(v1 - r[1]), std::fabs(v2 - r[2])));
                const double dm = std::fmax(std::fabs(v0 + r[0]), std::fmax(std::fabs(v1 + r[1]), std::fabs(v2 + r[2])));
                if (dp < 1e-9 || dm < 1e-9) found = (int)u;
            }
            if (found < 0) {
                found = (int)members.size();
                rep.push_back(i);
                rep.push_back(j);
                rb.push_back(v0);
                rb.push_back(v1);
                rb.push_back(v2);
                members.emplace_back();
            }
            members[found].push_back(b);
        }
    off.assign(1, 0);
    mem.clear();
    for (const auto &m : members) {
        mem.insert(mem.end(), m.begin(), m.end());
        off.push_back((int)mem.size());
    }
}

// W[f][u] = sum over the members pq of group u of |g_p(f) g_q(f)|^2
template <typename R>
__global__ void k_pc_group_w(DevGeom g, int U, const int *__restrict__ off, const int *__restrict__ mem,
                             const R *__restrict__ gains, R *__restrict__ W)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.F * U; e += gridDim.x * blockDim.x) {
        const int f = e / U, u = e % U;
        double a = 0.0;
        for (int m = off[u]; m < off[u + 1]; ++m) {
            const R *gi = gains + 2 * ((size_t)f * g.A + g.bl_i[mem[m]]), *gj = gains + 2 * ((size_t)f * g.A + g.bl_j[mem[m]]);
            a += (double)(gi[0] * gi[0] + gi[1] * gi[1]) * (double)(gj[0] * gj[0] + gj[1] * gj[1]);
        }
        W[e] = (R)a;
    }
}

// X[plane][u][pix] = sqrt(W_u) / sigma dOmega A K_u   (plane 0 = real, 1 = imag), K_u the
// fringe of the group's representative pair
template <typename R>
__global__ void k_pc_fringe(DevGeom g, int f, int t, int U, const int *__restrict__ rep, const R *__restrict__ W,
                            R *__restrict__ X)
{
    long long n = (long long)U * g.npix;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int u = (int)(e / g.npix), p = (int)(e % g.npix);
        int i = rep[2 * u], j = rep[2 * u + 1];
        R z2 = Tab<R>::za2(g)[(size_t)t * g.npix + p];
        R re = 0, im = 0;
        if (z2 >= R(0)) {
            // Gaussian beam from the squared zenith angle; the Airy beam from its table
            const R bm = g.beam32 ? (R)g.beam32[((size_t)f * g.T + t) * g.npix + p] : exp(Tab<R>::bcoef(g)[f] * z2);
            R w = sqrt(W[(size_t)f * U + u] * (R)g.inv_sigma2) * Tab<R>::domega(g)[p / g.R] * bm;
            R kr, ki;
            fringe(g, f, i, j, t, p, kr, ki);
            re = w * kr;
            im = w * ki;
        }
        X[e] = re;
        X[n + e] = im;
    }
}

// Reuse of the strided GEMM from k_simt.cu through a local copy (one TU each keeps
// the build parallel).
struct GemmArgsH {
    int M, N, K;
    long long sAb, sAi, sAk, sBb, sBk, sBj, sCb, sCi, sCj;
};

template <typename R>
__global__ void __launch_bounds__(256) k_gemm_h(GemmArgsH a, const R *__restrict__ A, const R *__restrict__ B,
                                                R *__restrict__ C)
{
    __shared__ R sA[16][65];
    __shared__ R sB[16][65];
    const long long b = blockIdx.z;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    R acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = R(0);
    const R *Ab = A + b * a.sAb;
    const R *Bb = B + b * a.sBb;
    for (int k0 = 0; k0 < a.K; k0 += 16) {
        for (int e = tid; e < 1024; e += 256) {
            int ii = e / 16, kk = e % 16;
            int gi = i0 + ii, gk = k0 + kk;
            sA[kk][ii] = (gi < a.M && gk < a.K) ? Ab[gi * a.sAi + gk * a.sAk] : R(0);
            int kb = e / 64, jj = e % 64;
            int gj = j0 + jj, gk2 = k0 + kb;
            sB[kb][jj] = (gj < a.N && gk2 < a.K) ? Bb[gk2 * a.sBk + gj * a.sBj] : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            R av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { av[q] = sA[kk][ty * 4 + q]; bv[q] = sB[kk][tx * 4 + q]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
        __syncthreads();
    }
    R *Cb = C + b * a.sCb;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int gi = i0 + ty * 4 + u, gj = j0 + tx * 4 + v;
            if (gi < a.M && gj < a.N) Cb[gi * a.sCi + gj * a.sCj] = acc[u][v];
        }
}

template <typename R>
static fm_status gemm_h(const GemmArgsH &a, long long batch, const R *A, const R *B, R *C, cudaStream_t st)
{
    while (batch > 0) {
        long long nb = batch > 65535 ? 65535 : batch;
        dim3 grid(cdiv(a.N, 64), cdiv(a.M, 64), (unsigned)nb);
        k_gemm_h<R><<<grid, 256, 0, st>>>(a, A, B, C);
        FM_CK_LAUNCH();
        A += nb * a.sAb; B += nb * a.sBb; C += nb * a.sCb;
        batch -= nb;
    }
    return FM_OK;
}

// acc64[j0][c][c'] += G[j0][c][c'] (blocks of channel f)
template <typename R>
__global__ void k_pc_accum(long long n, const R *__restrict__ G, double *__restrict__ acc)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        acc[e] += (double)G[e];
}

// diagonal: acc[k] += sum_{plane, b} S[plane][b][k]^2
template <typename R>
__global__ void k_pc_diag(int nk, int nrow, const R *__restrict__ S, double *__restrict__ acc)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < nrow; ++r) {
            double v = (double)S[(size_t)r * nk + k];
            s += v * v;
        }
        acc[k] += s;
    }
}

// S_pq(f) += |V_pq(f,t)|^2 over t (FP64, one thread per (f, pq))
template <typename R>
__global__ void k_pc_vis2(DevGeom g, const R *__restrict__ vis, double *__restrict__ s2)
{
    long long n = (long long)g.F * g.B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int f = (int)(e / g.B), b = (int)(e % g.B);
        double s = 0.0;
        for (int t = 0; t < g.T; ++t) {
            size_t o = (((size_t)f * g.T + t) * g.B + b) * 2;
            double vr = vis[o], vi = vis[o + 1];
            s += vr * vr + vi * vi;
        }
        s2[e] = s;
    }
}

// Gain block of Re(J^H J)/sigma^2 + diag(lam): parameters (a, k, c) with c = re/im.
// Same antenna: sum_f X_k X_k' delta_cc' sum_{pq ni a} |g_other|^2 S_pq;  antennas
// i < j of baseline pq: sum_f X_k X_k' Re(conj(u_c) u'_c' g_i g_j) S_pq with
// u = (1, i) for the first antenna and u' = (1, -i) for the conjugated second one.
template <typename R>
__global__ void k_pc_gain_block(DevGeom g, const double *__restrict__ s2, const R *__restrict__ gains,
                                const R *__restrict__ lam_gain, int have_prior, int dense, double *__restrict__ out)
{
    const int ng = 2 * g.A * g.NG;
    long long n = dense ? (long long)ng * ng : ng;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int r = dense ? (int)(e / ng) : (int)e, cidx = dense ? (int)(e % ng) : (int)e;
        int a1 = r / (2 * g.NG), k1 = (r / 2) % g.NG, c1 = r % 2;
        int a2 = cidx / (2 * g.NG), k2 = (cidx / 2) % g.NG, c2 = cidx % 2;
        double h = 0.0;
        if (a1 == a2) {
            if (c1 == c2) {
                for (int f = 0; f < g.F; ++f) {
                    double X = (double)Tab<R>::gleg(g)[f * g.NG + k1] * (double)Tab<R>::gleg(g)[f * g.NG + k2];
                    double d = 0.0;
                    for (int o = 0; o < g.A; ++o) {
                        if (o == a1) continue;
                        int b = o > a1 ? (a1 * g.A - a1 * (a1 + 1) / 2 + (o - a1 - 1)) : (o * g.A - o * (o + 1) / 2 + (a1 - o - 1));
                        double gr = gains[2 * (f * g.A + o)], gi = gains[2 * (f * g.A + o) + 1];
                        d += (gr * gr + gi * gi) * s2[(size_t)f * g.B + b];
                    }
                    h += X * d;
                }
            }
        } else {
            int i = a1 < a2 ? a1 : a2, j = a1 < a2 ? a2 : a1;
            int ci = a1 < a2 ? c1 : c2, cj = a1 < a2 ? c2 : c1;
            int ki = a1 < a2 ? k1 : k2, kj = a1 < a2 ? k2 : k1;
            int b = i * g.A - i * (i + 1) / 2 + (j - i - 1);
            for (int f = 0; f < g.F; ++f) {
                double X = (double)Tab<R>::gleg(g)[f * g.NG + ki] * (double)Tab<R>::gleg(g)[f * g.NG + kj];
                double gir = gains[2 * (f * g.A + i)], gii = gains[2 * (f * g.A + i) + 1];
                double gjr = gains[2 * (f * g.A + j)], gji = gains[2 * (f * g.A + j) + 1];
                double pr = gir * gjr - gii * gji, pi = gir * gji + gii * gjr;     // g_i g_j
                double v = (ci == 0 && cj == 0) ? pr : (ci == 1 && cj == 1) ? -pr : pi;
                h += X * v * s2[(size_t)f * g.B + b];
            }
        }
        h *= g.inv_sigma2;
        if (r == cidx && have_prior) h += (double)lam_gain[r];
        out[e] = h;
    }
}

// Cholesky of one block held in shared memory (n <= 64), FP64, with prior inflation:
// M = (H - diag(lam)) + c diag(lam), c = 1, 1.1, 1.21, ...  Writes L (lower) in R.
template <typename R>
__global__ void __launch_bounds__(64) k_pc_chol_small(int n, const double *__restrict__ H, const R *__restrict__ lam,
                                                      long long lam_off, int have_prior, R *__restrict__ L,
                                                      int *__restrict__ status)
{
    __shared__ double sM[64][65];
    __shared__ int bad;
    const int blk = blockIdx.x, tid = threadIdx.x;
    const double *Hb = H + (size_t)blk * n * n;
    double c = 1.0;
    for (int attempt = 0; attempt < 200; ++attempt) {
        for (int e = tid; e < n * n; e += blockDim.x) {
            int r = e / n, q = e % n;
            double v = Hb[e];
            if (r == q && have_prior) {
                double l = (double)lam[lam_off + (size_t)blk * n + r];
                v += (c - 1.0) * l;
            }
            sM[r][q] = v;
        }
        if (tid == 0) bad = 0;
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            if (tid == 0) {
                double d = sM[k][k];
                if (!(d > 0.0) || !isfinite(d)) bad = 1;
                sM[k][k] = bad ? 1.0 : sqrt(d);
            }
            __syncthreads();
            if (bad) break;
            double dk = sM[k][k];
            for (int r = k + 1 + tid; r < n; r += blockDim.x) sM[r][k] /= dk;
            __syncthreads();
            for (int r = k + 1 + tid; r < n; r += blockDim.x)
                for (int q = k + 1; q <= r; ++q) sM[r][q] -= sM[r][k] * sM[q][k];
            __syncthreads();
        }
        __syncthreads();
        if (!bad) break;
        c *= 1.1;
        __syncthreads();
        if (attempt == 199 && tid == 0) atomicExch(status, (int)FM_ERR_NOT_SPD);
    }
    R *Lb = L + (size_t)blk * n * n;
    for (int e = tid; e < n * n; e += blockDim.x) {
        int r = e / n, q = e % n;
        Lb[e] = (q <= r) ? (R)sM[r][q] : R(0);
    }
}

// Cholesky of the dense gain block in global FP64 scratch (one CTA), same inflation.
template <typename R>
__global__ void __launch_bounds__(256) k_pc_chol_big(int n, const double *__restrict__ H, const R *__restrict__ lam,
                                                     long long lam_off, int have_prior, double *__restrict__ W,
                                                     R *__restrict__ L, double *__restrict__ L64,
                                                     int *__restrict__ status)
{
    __shared__ int bad;
    const int tid = threadIdx.x;
    double c = 1.0;
    for (int attempt = 0; attempt < 200; ++attempt) {
        for (int e = tid; e < n * n; e += blockDim.x) {
            int r = e / n, q = e % n;
            double v = H[e];
            if (r == q && have_prior) v += (c - 1.0) * (double)lam[lam_off + r];
            W[e] = v;
        }
        if (tid == 0) bad = 0;
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            if (tid == 0) {
                double d = W[(size_t)k * n + k];
                if (!(d > 0.0) || !isfinite(d)) bad = 1;
                W[(size_t)k * n + k] = bad ? 1.0 : sqrt(d);
            }
            __syncthreads();
            if (bad) break;
            double dk = W[(size_t)k * n + k];
            for (int r = k + 1 + tid; r < n; r += blockDim.x) W[(size_t)r * n + k] /= dk;
            __syncthreads();
            long long m = (long long)(n - k - 1) * (n - k - 1);
            for (long long e = tid; e < m; e += blockDim.x) {
                int r = k + 1 + (int)(e / (n - k - 1)), q = k + 1 + (int)(e % (n - k - 1));
                if (q <= r) W[(size_t)r * n + q] -= W[(size_t)r * n + k] * W[(size_t)q * n + k];
            }
            __syncthreads();
        }
        __syncthreads();
        if (!bad) break;
        c *= 1.1;
        __syncthreads();
        if (attempt == 199 && tid == 0) atomicExch(status, (int)FM_ERR_NOT_SPD);
    }
    for (int e = tid; e < n * n; e += blockDim.x) {
        int r = e / n, q = e % n;
        L[e] = (q <= r) ? (R)W[e] : R(0);
        if (L64) L64[e] = (q <= r) ? W[e] : 0.0;
    }
}

// Inverse of the dense lower-triangular gain-block factor W (FP64, row-major): thread j
// solves W x = e_j by forward substitution in FP64 (x kept in Xd[j][.]), then stores
// Ginv[r][j] = x_r.  Used by the leapfrog's dense solves, which then become triangular
// matrix-vector products.  The gain block keeps FP64 throughout (factor, inverses, products):
// the global gain phase is held by the prior alone, so the block's condition number
// reaches 1e6 and a rounded inverse would misplace the data-constrained directions.
__global__ void __launch_bounds__(128) k_pc_tri_inv(int n, const double *__restrict__ W, double *__restrict__ Xd,
                                                    double *__restrict__ Ginv, double *__restrict__ GinvT)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double *x = Xd + (size_t)j * n;
        for (int r = 0; r < j; ++r) x[r] = 0.0;
        x[j] = 1.0 / W[(size_t)j * n + j];
        for (int r = j + 1; r < n; ++r) {
            const double *row = W + (size_t)r * n;
            double a = 0.0;
            for (int cc = j; cc < r; ++cc) a += row[cc] * x[cc];
            x[r] = -a / row[r];
        }
        for (int r = 0; r < n; ++r) {
            Ginv[(size_t)r * n + j] = x[r];
            GinvT[(size_t)j * n + r] = x[r];
        }
    }
}

// The gain block of the inverse mass matrix, Gm = L_g^-T L_g^-1 (symmetric), from the FP64
// inverse columns Xd[j][k] = (L_g^-1)[k][j]: Gm[r][c] = sum over k >= max(r, c) of
// Xd[r][k] Xd[c][k], in FP64.  A drift then needs one product with Gm.
__global__ void k_pc_gm(int n, const double *__restrict__ Xd, double *__restrict__ Gm)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        const double *xr = Xd + (size_t)r * n, *xc = Xd + (size_t)c * n;
        double a = 0.0;
        for (int k = r > c ? r : c; k < n; ++k) a += xr[k] * xc[k];
        Gm[e] = a;
    }
}

// Packed storage of a lower-triangular 64 x 64 block in 16-byte pieces of PER = 16 /
// sizeof(R) entries: row r keeps its first ceil((r + 1) / PER) pieces (entries past the
// diagonal in the last piece are zero), rows one after another.  With r = PER a + b, row r
// starts at piece PER a (a + 1) / 2 + b (a + 1); a block takes 544 pieces in FP32 and 1056 in
// FP64 instead of 1024, and every row starts on a 16-byte boundary.
template <typename R>
__host__ __device__ constexpr int tri_row_pieces(int r)
{
    return (r + (int)(16 / sizeof(R))) / (int)(16 / sizeof(R));
}
template <typename R>
__host__ __device__ constexpr int tri_row_start(int r)
{
    return (int)(16 / sizeof(R)) * (r / (int)(16 / sizeof(R))) * (r / (int)(16 / sizeof(R)) + 1) / 2 +
           (r % (int)(16 / sizeof(R))) * (r / (int)(16 / sizeof(R)) + 1);
}
template <typename R>
__host__ __device__ constexpr int tri_block_elems()
{
    return tri_row_start<R>(64) * (int)(16 / sizeof(R));
}
static_assert(tri_row_start<float>(64) == 544 && tri_row_start<double>(64) == 1056, "packed block size");
static_assert(tri_row_start<float>(5) == 6 && tri_row_start<float>(4) == 4, "packed row start");

// Inverses of the stored 64 x 64 sky-block factors (one CTA of 64 threads per block):
// the factor, as stored in the working type, is read into FP64 shared memory and thread
// j solves L x = e_j by forward substitution; Linv[r][j] = x_r, stored packed (above).
// Inverting the stored factor keeps L^-1 (L z) = z to FP64 rounding before the final store.
template <typename R>
__global__ void __launch_bounds__(64) k_pc_blk_inv(const R *__restrict__ L, R *__restrict__ Linv)
{
    extern __shared__ double sd[];
    double *sL = sd;                  // [64][65]
    double *sX = sd + 64 * 65;        // [64 columns][65]
    const R *Lb = L + (size_t)blockIdx.x * 4096;
    for (int e = threadIdx.x; e < 4096; e += 64) sL[(e >> 6) * 65 + (e & 63)] = (double)Lb[e];
    __syncthreads();
    const int j = threadIdx.x;
    double *x = sX + j * 65;
    for (int r = 0; r < 64; ++r) {
        double v = 0.0;
        if (r == j) v = 1.0 / sL[r * 65 + r];
        else if (r > j) {
            double a = 0.0;
            for (int cc = j; cc < r; ++cc) a += sL[r * 65 + cc] * x[cc];
            v = -a / sL[r * 65 + r];
        }
        x[r] = v;
    }
    R *Ib = Linv + (size_t)blockIdx.x * tri_block_elems<R>();
    constexpr int PER = 16 / sizeof(R);
    for (int r = 0; r < 64; ++r)
        if (j < tri_row_pieces<R>(r) * PER) Ib[tri_row_start<R>(r) * PER + j] = (R)x[r];
}

// Sky prior on the block diagonals: blocks[k/bs][k%bs][k%bs] += lam[k]
template <typename R>
__global__ void k_pc_add_prior(long long nsky, int bs, const R *__restrict__ lam, double *__restrict__ blocks)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nsky; k += (long long)gridDim.x * blockDim.x) {
        long long blk = k / bs;
        int c = (int)(k % bs);
        blocks[(size_t)blk * bs * bs + (size_t)c * bs + c] += (double)lam[k];
    }
}

// Diagonal mass matrix: L = sqrt(H_lik + c lam) with the same inflation rule.
template <typename R>
__global__ void k_pc_chol_diag(long long n, const double *__restrict__ H, const R *__restrict__ lam, int have_prior,
                               R *__restrict__ L, int *__restrict__ status)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double l = have_prior ? (double)lam[k] : 0.0;
        double v = H[k], c = 1.0;
        int a = 0;
        while (!(v > 0.0) && a < 200) { c *= 1.1; v = H[k] + (c - 1.0) * l; ++a; }
        if (!(v > 0.0) || !isfinite(v)) { atomicExch(status, (int)FM_ERR_NOT_SPD); v = 1.0; }
        L[k] = (R)sqrt(v);
    }
}

template <typename R>
fm_status run_build_precond(Ctx &c, const R *theta, int block, cudaStream_t st)
{
    const int bs = block;
    const int ng = 2 * c.A * c.NG;
    const long long nsky_blk = c.n_sky / bs;
    const long long sky_sz = nsky_blk * bs * bs;
    const long long gain_sz = bs > 1 ? (long long)ng * ng : ng;
    const long long need = sky_sz + gain_sz;
    if (c.pc_size != need || c.pc_block != bs) {
        // (re)allocate: previous buffers stay in c.allocs until destroy
        double *blocks = nullptr;
        if (cudaMalloc(&blocks, sizeof(double) * need) != cudaSuccess) { set_error("cudaMalloc precond"); return FM_ERR_ALLOC; }
        c.allocs.push_back(blocks);
        void *chol = nullptr;
        if (cudaMalloc(&chol, c.rsz * need) != cudaSuccess) { set_error("cudaMalloc precond factors"); return FM_ERR_ALLOC; }
        c.allocs.push_back(chol);
        c.pc_blocks = blocks;
        c.pc_chol = chol;
        c.pc_size = need;
        c.pc_block = bs;
    }
    // baseline groups (once per handle)
    if (!c.pc_grp) {
        std::vector<int> rep, off, mem;
        pc_groups(c, rep, off, mem);
        c.pc_U = (int)off.size() - 1;
        std::vector<int> all(rep);
        all.insert(all.end(), off.begin(), off.end());
        all.insert(all.end(), mem.begin(), mem.end());
        void *d = nullptr;
        if (cudaMalloc(&d, sizeof(int) * all.size()) != cudaSuccess) { set_error("cudaMalloc precond groups"); return FM_ERR_ALLOC; }
        c.allocs.push_back(d);
        FM_CK(cudaMemcpy(d, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
        c.pc_grp = static_cast<int *>(d);
    }
    const int U = c.pc_U;
    const int *g_rep = c.pc_grp, *g_off = c.pc_grp + 2 * U, *g_mem = g_off + U + 1;
    // scratch for TB LSTs of one channel: fringes X [TB][2][U][npix], Q [2][U][D][M] (CUDA-core
    // route only), S [TB][2][U][nk], G [nk/bs][bs][bs], group weights W [F][U].  The tensor-core
    // transform takes TB LSTs' response maps per launch.
    const bool tcx = std::is_same<R, float>::value && c.mtc.on;
    const int TB = tcx ? (c.T < 4 ? c.T : 4) : 1;
    size_t nX = 2 * (size_t)U * c.npix * TB, nQ = tcx ? 0 : 2 * (size_t)U * c.D * c.M, nS = 2 * (size_t)U * c.nk * TB;
    // (counts rounded up to even so that the FP64 scratch after them stays 8-byte aligned)
    size_t nG = ((size_t)c.nk * bs + 1) & ~(size_t)1, nW = ((size_t)c.F * U + 1) & ~(size_t)1;
    R *X = nullptr;
    size_t scratch = (nX + nQ + nS + nG + nW) * sizeof(R) + sizeof(double) * ((size_t)c.F * c.B + (size_t)ng * ng);
    if (cudaMalloc(&X, scratch) != cudaSuccess) { set_error("cudaMalloc precond scratch (%zu bytes)", scratch); return FM_ERR_ALLOC; }
    R *Q = X + nX, *S = Q + nQ, *G = S + nS, *Wg = G + nG;
    double *s2 = reinterpret_cast<double *>(Wg + nW);
    double *W = s2 + (size_t)c.F * c.B;
    fm_status rc = FM_OK;
    do {
        R *gn = (R *)c.gains;
        R *x = (R *)c.x, *vis = (R *)c.vis;
        if ((rc = launch_gains<R>(c, theta + c.n_sky, gn, st)) != FM_OK) break;
        if (cudaMemsetAsync(c.pc_blocks, 0, sizeof(double) * need, st) != cudaSuccess) { rc = FM_ERR_CUDA; break; }
        k_pc_group_w<R><<<cdiv((long long)c.F * U, 256), 256, 0, st>>>(c.g, U, g_off, g_mem, gn, Wg);
        if (c.K > 0 && c.pc_gacc_n < (size_t)c.nk * bs) {
            // (re)allocate for this block size: a previous buffer stays in c.allocs until destroy
            if (cudaMalloc(&c.pc_gacc, sizeof(double) * (size_t)c.nk * bs) != cudaSuccess) {
                c.pc_gacc = nullptr;
                c.pc_gacc_n = 0;
                rc = FM_ERR_ALLOC;
                set_error("cudaMalloc precond channel blocks");
                break;
            }
            c.allocs.push_back(c.pc_gacc);
            c.pc_gacc_n = (size_t)c.nk * bs;
        }
        for (int f = 0; f < c.F && rc == FM_OK; ++f) {
            // Legendre-in-frequency compression: the channel's blocks are summed apart, then
            // spread into the K compressed parameters' blocks with the weights X_k(nu_f)^2
            double *accf = c.K > 0 ? c.pc_gacc : c.pc_blocks + (size_t)f * c.nk * bs;
            if (c.K > 0 && cudaMemsetAsync(accf, 0, sizeof(double) * (size_t)c.nk * bs, st) != cudaSuccess) {
                rc = FM_ERR_CUDA;
                break;
            }
            for (int t = 0; t < c.T; t += TB) {
                const int tbn = c.T - t < TB ? c.T - t : TB;
                for (int tb = 0; tb < tbn; ++tb)
                    k_pc_fringe<R><<<2048, 256, 0, st>>>(c.g, f, t + tb, U, g_rep, Wg, X + (size_t)tb * 2 * U * c.npix);
                if (cudaGetLastError() != cudaSuccess) { rc = FM_ERR_CUDA; break; }
                if (tcx) {
                    // S[tb,pl,b][m][n] = sum_{d,r} Phi[r][m] X[tb,pl,b][d][r] P[d][n]: the tensor-core
                    // pixel -> mode transform over the 2U response maps of tbn LSTs
                    if ((rc = launch_modes_tc_adjoint_maps(c, (const float *)X, 2 * U * tbn, (float *)S, st)) != FM_OK)
                        break;
                } else {
                    // Q[pl,b][d][m] = sum_r X[pl,b][d][r] Phi[r][m]
                    const R *phi = std::is_same<R, float>::value ? (const R *)c.g.phi32 : (const R *)c.g.phi64;
                    const R *leg = std::is_same<R, float>::value ? (const R *)c.g.leg32 : (const R *)c.g.leg64;
                    GemmArgsH q1{(int)(2LL * U * c.D), c.M, c.R, 0, c.R, 1, 0, c.M, 1, 0, c.M, 1};
                    if ((rc = gemm_h<R>(q1, 1, X, phi, Q, st)) != FM_OK) break;
                    // S[pl,b][m][n] = sum_d Q[pl,b][d][m] P[d][n]
                    GemmArgsH q2{c.M, c.N, c.D, (long long)c.D * c.M, 1, c.M, 0, c.N, 1, c.nk, c.N, 1};
                    if ((rc = gemm_h<R>(q2, 2LL * U, Q, leg, S, st)) != FM_OK) break;
                }
                if (bs > 1) {
                    // G[j0][c][c'] = sum_{tb,pl,b} S[tb,pl,b][j0*bs+c] S[tb,pl,b][j0*bs+c']
                    GemmArgsH q3{bs, bs, 2 * U * tbn, bs, 1, c.nk, bs, c.nk, 1, (long long)bs * bs, bs, 1};
                    if ((rc = gemm_h<R>(q3, c.nk / bs, S, S, G, st)) != FM_OK) break;
                    k_pc_accum<R><<<512, 256, 0, st>>>((long long)c.nk * bs, G, accf);
                } else {
                    k_pc_diag<R><<<cdiv(c.nk, 256), 256, 0, st>>>(c.nk, 2 * U * tbn, S, accf);
                }
                if (cudaGetLastError() != cudaSuccess) { rc = FM_ERR_CUDA; break; }
            }
            if (rc == FM_OK && c.K > 0) rc = launch_freq_spread(c, f, (long long)c.nk * bs, accf, c.pc_blocks, st);
        }
        if (rc != FM_OK) break;
        // prior on the sky diagonal
        // (added by the Cholesky kernels' inflation logic through H + lam; store H + lam here)
        // gain block: needs V at theta
        const R *sky = theta;
        if (c.K > 0) {
            if ((rc = launch_freq_expand<R>(c, theta, (R *)c.ax, st)) != FM_OK) break;
            sky = (const R *)c.ax;
        }
        if ((rc = vis_of_modes<R>(c, sky, x, vis, st)) != FM_OK) break;
        k_pc_vis2<R><<<cdiv((long long)c.F * c.B, 256), 256, 0, st>>>(c.g, vis, s2);
        k_pc_gain_block<R><<<512, 256, 0, st>>>(c.g, s2, gn, c.have_prior ? (const R *)c.lam + c.n_sky : nullptr, c.have_prior ? 1 : 0, bs > 1 ? 1 : 0,
                                                c.pc_blocks + sky_sz);
        if (c.have_prior)
            k_pc_add_prior<R><<<cdiv(c.n_sky, 256), 256, 0, st>>>(c.n_sky, bs, (const R *)c.lam, c.pc_blocks);
        if (cudaGetLastError() != cudaSuccess) { rc = FM_ERR_CUDA; break; }
        // factorise every block (prior inflation on failure)
        R *Lf = (R *)c.pc_chol;
        if (bs > 1) {
            k_pc_chol_small<R><<<(unsigned)nsky_blk, 64, 0, st>>>(bs, c.pc_blocks, (const R *)c.lam, 0,
                                                                  c.have_prior ? 1 : 0, Lf, c.status);
            if (ng > 0 && !c.pc_ginv) {
                if (cudaMalloc(&c.pc_ginv, 4 * sizeof(double) * (size_t)ng * ng) != cudaSuccess ||
                    cudaMalloc(&c.pc_tmp, sizeof(double) * (size_t)ng * ng) != cudaSuccess) {
                    rc = FM_ERR_ALLOC;
                    set_error("cudaMalloc gain-block inverse");
                    break;
                }
                c.allocs.push_back(c.pc_ginv);
                c.allocs.push_back(c.pc_tmp);
            }
            // FP64 gain block: [0] L_g, [1] L_g^-1, [2] L_g^-T, [3] L_g^-T L_g^-1
            double *G64 = (double *)c.pc_ginv;
            k_pc_chol_big<R><<<1, 256, 0, st>>>(ng, c.pc_blocks + sky_sz, (const R *)c.lam, c.n_sky,
                                                c.have_prior ? 1 : 0, W, Lf + sky_sz, G64, c.status);
            if (!c.pc_linv) {
                if (cudaMalloc(&c.pc_linv, sizeof(R) * (size_t)nsky_blk * tri_block_elems<R>()) != cudaSuccess) {
                    rc = FM_ERR_ALLOC;
                    set_error("cudaMalloc sky-block inverses");
                    break;
                }
                c.allocs.push_back(c.pc_linv);
            }
            smem_opt_in(k_pc_blk_inv<R>);
            k_pc_blk_inv<R><<<(unsigned)nsky_blk, 64, 2 * 64 * 65 * sizeof(double), st>>>(Lf, (R *)c.pc_linv);
            if (ng > 0) {
                k_pc_tri_inv<<<cdiv(ng, 128), 128, 0, st>>>(ng, W, c.pc_tmp, G64 + (size_t)ng * ng,
                                                            G64 + 2 * (size_t)ng * ng);
                k_pc_gm<<<cdiv((long long)ng * ng, 256), 256, 0, st>>>(ng, c.pc_tmp, G64 + 3 * (size_t)ng * ng);
            }
        } else {
            k_pc_chol_diag<R><<<cdiv(need, 256), 256, 0, st>>>(need, c.pc_blocks, (const R *)c.lam,
                                                               c.have_prior ? 1 : 0, Lf, c.status);
        }
        if (cudaGetLastError() != cudaSuccess) { rc = FM_ERR_CUDA; break; }
    } while (0);
    if (rc == FM_OK) rc = FM_OK;
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(X);
    if (rc != FM_OK) { set_error("precond build failed (%d)", (int)rc); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "precond build", __FILE__, __LINE__);
    int stv = 0;
    FM_CK(cudaMemcpy(&stv, c.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (stv == FM_ERR_NOT_SPD) {
        FM_CK(cudaMemset(c.status, 0, sizeof(int)));
        set_error("a preconditioner block stayed indefinite after 200 prior inflations");
        return FM_ERR_NOT_SPD;
    }
    return FM_OK;
}

// ------------------------------------------------------------------ leapfrog
__global__ void k_set_lf_params(double *prm, double eps, double u)
{
    prm[0] = eps;
    prm[1] = u;
}

template <typename R>
__global__ void k_copy(long long n, const R *__restrict__ x, R *__restrict__ y)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        y[k] = x[k];
}

// Block-diagonal triangular algebra of the mass-matrix factor M = L L^T (App. B):
// v = in; if (fwd) v = L^-1 v (forward substitution; kin[blk] = sum v^2 in FP64);
// if (bwd) v = L^-T v (backward substitution); then q += eps v (q != NULL) and/or
// out = v (out != NULL).  mul: out = L in instead.  Arithmetic in the working type R.
//
// The solves use the explicit inverses of the factors (computed in FP64 from the stored
// factors when the preconditioner is built), so every operation is a triangular
// matrix-vector product without a serial dependency.  One warp per 64 x 64 sky block:
// the block is copied to shared memory with cp.async in 16-byte pieces (L^-1 packed as it
// is stored, 8.7 KB in FP32, so that twice as many warps fit on an SM; L, stored full, for
// mul into an XOR-permuted image), lane l owns entries l and l + 32, and the vector is read
// from shared memory.  The dense gain block follows in k_lf_dense.
constexpr int LF_WARPS = 4;

// shared bytes of one warp of k_lf_tri: the block image, the vector, an mbarrier and a flag
template <typename R>
__host__ __device__ constexpr size_t lf_warp_bytes(int mul)
{
    return sizeof(R) * (size_t)((mul ? 4096 : tri_block_elems<R>()) + 64) + 16;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename R>
__device__ __forceinline__ R warp_sum(R a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// y = T v for a 64 x 64 lower-triangular T stored with zeros above the diagonal in the
// image S (row-major, the 16-byte pieces of row r permuted by XOR with r mod pieces per row,
// so that a row read touches no bank twice): lane l forms rows l and l + 32 from whole
// 16-byte pieces of its rows and broadcast pieces of v (vs, shared)
template <typename R>
__device__ __forceinline__ void lower_mv(const R *S, const R *vs, R &y0, R &y1)
{
    constexpr int PER = 16 / sizeof(R), NP = 64 / PER;
    const int lane = threadIdx.x & 31;
    const R *r0 = S + lane * 64, *r1 = S + (lane + 32) * 64;
    const int x0 = lane & (NP - 1);
    R a0 = 0, a1 = 0;
#pragma unroll
    for (int pc = 0; pc < NP; ++pc) {
        const int ph = (pc ^ x0) * PER;              // rows l and l + 32 share the permutation
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const R vq = vs[pc * PER + q];
            a0 += r0[ph + q] * vq;
            a1 += r1[ph + q] * vq;
        }
    }
    y0 = a0;
    y1 = a1;
}

// The same product for T in the packed form (tri_row_start): lane l reads only the stored
// pieces of rows l and l + 32, in the order of lower_mv, so the sums are the same
template <typename R>
__device__ __forceinline__ void lower_mv_packed(const R *P, const R *vs, R &y0, R &y1)
{
    constexpr int PER = 16 / sizeof(R), NP = 64 / PER;
    struct alignas(16) Piece { R v[PER]; };
    const int lane = threadIdx.x & 31;
    const Piece *r0 = reinterpret_cast<const Piece *>(P) + tri_row_start<R>(lane);
    const Piece *r1 = reinterpret_cast<const Piece *>(P) + tri_row_start<R>(lane + 32);
    const int n0 = tri_row_pieces<R>(lane), n1 = tri_row_pieces<R>(lane + 32);
    R a0 = 0, a1 = 0;
#pragma unroll
    for (int pc = 0; pc < NP; ++pc) {
        if (pc < n0) {
            const Piece t = r0[pc];
#pragma unroll
            for (int q = 0; q < PER; ++q) a0 += t.v[q] * vs[pc * PER + q];
        }
        if (pc < n1) {
            const Piece t = r1[pc];
#pragma unroll
            for (int q = 0; q < PER; ++q) a1 += t.v[q] * vs[pc * PER + q];
        }
    }
    y0 = a0;
    y1 = a1;
}

// Dense gain block of the mass-matrix algebra: y_r = sum over c <= r (lower) or c >= r
// (upper) of M[r][c] x_c with M = L_g, L_g^-1 or L_g^-T (row-major), one warp per row so
// that all rows' loads are in flight together.  Outputs: y (scratch), kin[r] = y_r^2,
// q[r] += eps y_r, out[r] = y_r (each when non-NULL).
template <typename R, typename X>
__global__ void __launch_bounds__(256) k_lf_dense(int n, const double *__restrict__ M, int lower,
                                                  const X *__restrict__ x, double *__restrict__ y, double *__restrict__ kin,
                                                  R *__restrict__ q, const double *__restrict__ peps,
                                                  R *__restrict__ out)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= n) return;
    const double eps = q ? *peps : 0.0;
    const double *row = M + (size_t)r * n;
    double a = 0;
    for (int cc = lane; cc < n; cc += 32)
        if (lower ? cc <= r : cc >= r) a += row[cc] * (double)x[cc];
    a = warp_sum(a);
    if (lane == 0) {
        if (y) y[r] = a;
        if (kin) kin[r] = a * a;
        if (q) q[r] += (R)(eps * a);
        if (out) out[r] = (R)a;
    }
}

// The dense gain block as the first nctas CTAs of k_lf_tri (so that they run in its first
// wave): one warp per row r of the n x n row-major matrix M (mode 0: entries c >= r, 1: c <= r,
// 2: all), x = in + base, each lane taking c = lane, lane + 32, ... as k_lf_dense does;
// outputs at base + r and the kinetic partial kin[r] = y_r^2 (when kin != NULL).
template <typename R>
struct LfDense {
    const double *M;                  // FP64 (the gain block keeps FP64 throughout)
    int n, mode;
    long long base;
    unsigned nctas;
    double *kin;
};

template <typename R>
__global__ void __launch_bounds__(LF_WARPS * 32) k_lf_tri(long long nblk, const R *__restrict__ Li,
                                                          const R *__restrict__ L, const R *__restrict__ in, int fwd,
                                                          int bwd, int mul, R *__restrict__ q,
                                                          const double *__restrict__ peps,
                                                          R *__restrict__ out, double *__restrict__ kin,
                                                          LfDense<R> dn, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const double eps = q ? *peps : 0.0;
    if (blockIdx.x < dn.nctas) {
        // ------------------------------------------------ dense gain rows, one warp per row
        const int r = (int)blockIdx.x * LF_WARPS + w;
        if (r >= dn.n) return;
        const double *row = dn.M + (size_t)r * dn.n;
        const R *x = in + dn.base;
        double a = 0;
        for (int cc = lane; cc < dn.n; cc += 32)
            if (dn.mode == 2 || (dn.mode == 1 ? cc <= r : cc >= r)) a += row[cc] * (double)x[cc];
        a = warp_sum(a);
        if (lane == 0) {
            if (dn.kin) dn.kin[r] = a * a;
            if (q && !mul) q[dn.base + r] += (R)(eps * a);
            if (out) out[dn.base + r] = (R)a;
        }
        return;
    }
    {
        // ------------------------------------------------ one 64 x 64 block per warp
        const long long blk = (long long)(blockIdx.x - dn.nctas) * LF_WARPS + w;
        if (blk >= nblk) return;
        constexpr int PER = 16 / sizeof(R), NP = 64 / PER;     // elements per 16-byte piece, pieces per row
        const int wsz = mul ? 4096 : tri_block_elems<R>();      // block image, then the 64-vector
        // per warp: the image, the vector, an mbarrier and an abort flag
        unsigned char *wb = smem_raw + (size_t)w * lf_warp_bytes<R>(mul);
        R *S = reinterpret_cast<R *>(wb);
        R *vs = S + wsz;
        const uint32_t bar = tc::su32(wb + sizeof(R) * (wsz + 64));
        volatile int *wabort = reinterpret_cast<volatile int *>(wb + sizeof(R) * (wsz + 64) + 8);
        const long long off = blk * 64;
        if (mul) {                                      // the factor, stored full: XOR-permuted image
            const R *Lb = L + blk * 4096;
            for (int e = lane; e < 64 * NP; e += 32) {
                const int r = e / NP, pc = e % NP;
                cp_async16(S + r * 64 + ((pc ^ (r & (NP - 1))) * PER), Lb + r * 64 + pc * PER);
            }
            vs[lane] = in[off + lane];
            vs[lane + 32] = in[off + lane + 32];
            cp_async_wait_all();
        } else {                                        // its inverse, packed: one bulk copy as it is stored
            constexpr uint32_t bytes = (uint32_t)(sizeof(R) * tri_block_elems<R>());
            if (lane == 0) {
                *wabort = 0;
                tc::mbar_init(bar, 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                tc::mbar_expect_tx(bar, bytes);
                tc::bulk_g2s(tc::su32(S), Li + blk * tri_block_elems<R>(), bytes, bar);
            }
            vs[lane] = in[off + lane];
            vs[lane + 32] = in[off + lane + 32];
            __syncwarp();
            if (!tc::mbar_wait_ab(bar, 0u, wabort)) {
                if (lane == 0) atomicExch(status, (int)FM_ERR_TIMEOUT);
                return;
            }
        }
        __syncwarp();
        if (mul) {
            R y0, y1;
            lower_mv<R>(S, vs, y0, y1);
            out[off + lane] = y0;
            out[off + lane + 32] = y1;
            return;
        }
        R v0 = vs[lane], v1 = vs[lane + 32];
        if (fwd) {
            lower_mv_packed<R>(S, vs, v0, v1);
            if (kin) {
                double sq = warp_sum((double)v0 * (double)v0 + (double)v1 * (double)v1);
                if (lane == 0) kin[blk] = sq;
            }
        }
        if (bwd) {
            // v = T^T v: lane l forms entries l and l + 32 from the rows r that store them
            // (consecutive entries of row r across the lanes)
            __syncwarp();
            vs[lane] = v0;
            vs[lane + 32] = v1;
            __syncwarp();
            R b0 = 0, b1 = 0;
#pragma unroll
            for (int r = 0; r < 64; ++r) {
                const R zr = vs[r];
                const R *row = S + tri_row_start<R>(r) * PER;
                const int len = tri_row_pieces<R>(r) * PER;
                if (lane < len) b0 += row[lane] * zr;
                if (lane + 32 < len) b1 += row[lane + 32] * zr;
            }
            v0 = b0;
            v1 = b1;
        }
        if (q) { q[off + lane] += (R)(eps * v0); q[off + lane + 32] += (R)(eps * v1); }
        if (out) { out[off + lane] = v0; out[off + lane + 32] = v1; }
        return;
    }
}

// Diagonal mass matrix (block = 1): the same operations elementwise with l = L[k].
template <typename R>
__global__ void __launch_bounds__(256) k_lf_solve_diag(long long n, const R *__restrict__ L, const R *__restrict__ in,
                                                       int fwd, int bwd, int mul, R *__restrict__ q,
                                                       const double *__restrict__ peps,
                                                       R *__restrict__ out, double *__restrict__ kin)
{
    __shared__ double red[256];
    double s = 0.0;
    const double eps = q ? *peps : 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double l = (double)L[k];
        double v = (double)in[k];
        if (mul) { out[k] = (R)(v * l); continue; }
        if (fwd) { v /= l; s += v * v; }
        if (bwd) v /= l;
        if (q) q[k] += (R)(eps * v);
        if (out) out[k] = (R)v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && kin) kin[blockIdx.x] = red[0];
}

// out = half the sum of part[0 .. n) in a fixed order: thread t adds the elements t + 1024 j in
// four interleaved running sums (four loads in flight), then the threads' sums pairwise
constexpr int SUM_THREADS = 1024;
__global__ void __launch_bounds__(SUM_THREADS) k_sum_to(int n, const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double red[SUM_THREADS];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = threadIdx.x; i0 < n; i0 += 4 * SUM_THREADS) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * SUM_THREADS;
            v[u] = i < n ? part[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] += v[u];
    }
    red[threadIdx.x] = (s[0] + s[1]) + (s[2] + s[3]);
    __syncthreads();
    for (int w = SUM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * red[0];
}

// H0 = U0 + K0, H1 = U1 + K1, accept iff u < exp(H0 - H1); non-finite -> reject.
__global__ void k_lf_finish(const double *__restrict__ sc, const double *__restrict__ prm, double *__restrict__ h_out,
                            int *__restrict__ acc,
                            int *__restrict__ status)
{
    double H0 = sc[0] + sc[2], H1 = sc[1] + sc[3];
    h_out[0] = H0;
    h_out[1] = H1;
    int a;
    if (!isfinite(H0) || !isfinite(H1)) {
        a = 0;
        atomicExch(status, (int)FM_ERR_NONFINITE);
    } else {
        a = (H1 <= H0) ? 1 : (prm[1] < exp(H0 - H1) ? 1 : 0);
    }
    *acc = a;
}

template <typename R>
__global__ void k_lf_restore(long long n, const int *__restrict__ acc, const R *__restrict__ q0, R *__restrict__ q)
{
    if (*acc) return;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        q[k] = q0[k];
}

template <typename R>
static fm_status lf_blocks(Ctx &c, const R *in, int fwd, int bwd, int mul, R *q, const double *peps, R *out,
                           double *kin_out, cudaStream_t st)
{
    const int bs = c.pc_block;
    const R *L = (const R *)c.pc_chol;
    double *part = c.lf_scal + 8;
    if (bs > 1) {
        const long long nb = c.n_sky / bs;
        const int ng = 2 * c.A * c.NG;
        const size_t smem = (size_t)LF_WARPS * lf_warp_bytes<R>(mul);
        FM_CK(smem_opt_in(k_lf_tri<R>));
        const long long grid = (nb + LF_WARPS - 1) / LF_WARPS;
        // the gain block runs as extra warps of the same launch: one FP64 product with L_g (mul),
        // L_g^-1 (fwd), L_g^-T (bwd) or L_g^-T L_g^-1 (fwd and bwd, no kinetic energy)
        const double *G64 = (const double *)c.pc_ginv, *Gi = G64 + (size_t)ng * ng;
        LfDense<R> dn{nullptr, ng, 0, c.n_sky, 0u, nullptr};
        if (ng > 0) {
            if (mul) { dn.M = G64; dn.mode = 1; }
            else if (fwd && bwd) { if (!kin_out) { dn.M = Gi + 2 * (size_t)ng * ng; dn.mode = 2; } }
            else if (fwd) { dn.M = Gi; dn.mode = 1; dn.kin = kin_out ? part + nb : nullptr; }
            else if (bwd) { dn.M = Gi + (size_t)ng * ng; dn.mode = 0; }
        }
        if (dn.M) dn.nctas = cdiv(ng, LF_WARPS);
        const long long gtot = grid + dn.nctas;
        k_lf_tri<R><<<(unsigned)gtot, LF_WARPS * 32, smem, st>>>(nb, (const R *)c.pc_linv, L, in, fwd, bwd, mul, q,
                                                                peps, out, kin_out ? part : nullptr, dn, c.status);
        FM_CK_LAUNCH();
        if (ng > 0 && !dn.M && fwd && bwd) {     // both solves with the kinetic energy: two products
            const long long base = c.n_sky;
            const unsigned dg = cdiv(ng, 8);
            double *y = (double *)c.lf_y;
            k_lf_dense<R, R><<<dg, 256, 0, st>>>(ng, Gi, 1, in + base, y, part + nb, nullptr, peps, nullptr);
            FM_CK_LAUNCH();
            k_lf_dense<R, double><<<dg, 256, 0, st>>>(ng, Gi + (size_t)ng * ng, 0, y, nullptr, nullptr,
                                              q ? q + base : nullptr, peps, out ? out + base : nullptr);
            FM_CK_LAUNCH();
        }
        if (kin_out) {
            k_sum_to<<<1, SUM_THREADS, 0, st>>>((int)(nb + ng), part, kin_out);
            FM_CK_LAUNCH();
        }
    } else {
        k_lf_solve_diag<R><<<512, 256, 0, st>>>(c.n_par, L, in, fwd, bwd, mul, q, peps, out, kin_out ? part : nullptr);
        FM_CK_LAUNCH();
        if (kin_out) {
            k_sum_to<<<1, SUM_THREADS, 0, st>>>(512, part, kin_out);
            FM_CK_LAUNCH();
        }
    }
    return FM_OK;
}

template <typename R>
static fm_status lf_ensure(Ctx &c)
{
    if (c.lf_q0) return FM_OK;
    const long long n = c.n_par;
    if (cudaMalloc(&c.lf_q0, c.rsz * n) != cudaSuccess || cudaMalloc(&c.lf_g, c.rsz * n) != cudaSuccess) {
        set_error("cudaMalloc leapfrog state");
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(c.lf_q0);
    c.allocs.push_back(c.lf_g);
    const long long nb = c.n_sky + 1024;
    if (cudaMalloc(&c.lf_scal, sizeof(double) * (8 + nb)) != cudaSuccess) {
        set_error("cudaMalloc leapfrog scalars");
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(c.lf_scal);
    if (cudaMalloc(&c.lf_y, sizeof(double) * (size_t)(2 * c.A * c.NG + 1)) != cudaSuccess) {
        set_error("cudaMalloc leapfrog scratch");
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(c.lf_y);
    if (cudaMalloc(&c.lf_prm, sizeof(double) * 2) != cudaSuccess) {
        set_error("cudaMalloc leapfrog parameters");
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(c.lf_prm);
    return FM_OK;
}

// kinetic energy K = z.z/2 (L z = p) into *kin_out; with q != NULL also q += eps L^-T z,
// eps = *peps (device)
template <typename R>
static fm_status lf_kinetic_drift(Ctx &c, const R *p, R *q, const double *peps, double *kin_out, cudaStream_t st)
{
    return lf_blocks<R>(c, p, 1, q ? 1 : 0, 0, q, peps, nullptr, kin_out, st);
}

template <typename R>
fm_status run_precond_apply(Ctx &c, int op, const R *in, R *out, cudaStream_t st)
{
    FM_TRY(lf_ensure<R>(c));
    switch (op) {
    case 0: return lf_blocks<R>(c, in, 0, 0, 1, nullptr, nullptr, out, nullptr, st);
    case 1: return lf_blocks<R>(c, in, 1, 0, 0, nullptr, nullptr, out, nullptr, st);
    case 2: return lf_blocks<R>(c, in, 0, 1, 0, nullptr, nullptr, out, nullptr, st);
    case 3: return lf_blocks<R>(c, in, 1, 1, 0, nullptr, nullptr, out, nullptr, st);
    default: set_error("op must be 0..3"); return FM_ERR_INVALID_ARG;
    }
}
template fm_status run_precond_apply<float>(Ctx &, int, const float *, float *, cudaStream_t);
template fm_status run_precond_apply<double>(Ctx &, int, const double *, double *, cudaStream_t);

// One trajectory: the kernels read eps = prm[0] and the accept uniform u = prm[1] from device
// memory (a captured trajectory is replayed with new values by rewriting prm).
template <typename R>
fm_status run_leapfrog(Ctx &c, R *q, R *p, const double *prm, int n_steps, double *h_out, int *acc_out,
                       cudaStream_t st)
{
    const long long n = c.n_par;
    FM_TRY(lf_ensure<R>(c));
    R *q0 = (R *)c.lf_q0, *g = (R *)c.lf_g;
    double *sc = c.lf_scal;            // U0, U1, K0, K1, chi2
    if (n_steps < 1) {
        set_error("n_steps must be at least 1");
        return FM_ERR_INVALID_ARG;
    }
    k_copy<R><<<512, 256, 0, st>>>(n, q, q0);
    FM_CK_LAUNCH();
    FM_TRY(lf_kinetic_drift<R>(c, p, nullptr, nullptr, sc + 2, st));     // K0, before any kick
    // every gradient evaluation ends with the kick that uses its gradient, fused into its last
    // pass: a half kick after the first and the last, and between steps one full kick (the
    // closing half kick of a step and the opening one of the next use the same gradient)
    FM_TRY(run_chi2_grad<R>(c, q, sc + 4, sc + 0, g, st, p, prm, 0.5));
    for (int s = 0; s < n_steps; ++s) {
        FM_TRY(lf_kinetic_drift<R>(c, p, q, prm, nullptr, st));
        FM_TRY(run_chi2_grad<R>(c, q, sc + 4, sc + 1, g, st, p, prm, s + 1 < n_steps ? 1.0 : 0.5));
    }
    FM_TRY(lf_kinetic_drift<R>(c, p, nullptr, nullptr, sc + 3, st));
    k_lf_finish<<<1, 1, 0, st>>>(sc, prm, h_out, acc_out, c.status);
    FM_CK_LAUNCH();
    k_lf_restore<R><<<512, 256, 0, st>>>(n, acc_out, q0, q);
    FM_CK_LAUNCH();
    return FM_OK;
}

// the per-handle parameter slot written in stream order (fm_leapfrog)
template <typename R>
fm_status set_leapfrog_params(Ctx &c, double eps, double u, cudaStream_t st)
{
    FM_TRY(lf_ensure<R>(c));
    k_set_lf_params<<<1, 1, 0, st>>>(c.lf_prm, eps, u);
    FM_CK_LAUNCH();
    return FM_OK;
}
template fm_status set_leapfrog_params<float>(Ctx &, double, double, cudaStream_t);
template fm_status set_leapfrog_params<double>(Ctx &, double, double, cudaStream_t);

// allocations a trajectory needs, made outside any stream capture
template <typename R>
fm_status prepare_leapfrog(Ctx &c)
{
    return lf_ensure<R>(c);
}
template fm_status prepare_leapfrog<float>(Ctx &);
template fm_status prepare_leapfrog<double>(Ctx &);

template fm_status run_leapfrog<float>(Ctx &, float *, float *, const double *, int, double *, int *, cudaStream_t);
template fm_status run_leapfrog<double>(Ctx &, double *, double *, const double *, int, double *, int *, cudaStream_t);

template fm_status run_build_precond<float>(Ctx &, const float *, int, cudaStream_t);
template fm_status run_build_precond<double>(Ctx &, const double *, int, cudaStream_t);

}  // namespace fm
