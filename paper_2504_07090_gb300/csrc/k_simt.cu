// CUDA-core kernels of the forward model and its adjoint, templated on the real type
// (double for the complex128 path, float for the plain FP32 path):
//   - separable mode <-> pixel transforms (Eq. fg_separable) as strided batched GEMMs;
//   - antenna phasors E_ip = exp(-2 pi i nu r_i . s_p / c) generated in-kernel, never
//     stored (b_pq = r_p - r_q makes K_pq = E_p conj(E_q), Eq. rime_discrete);
//   - the fringe contraction V_pq = sum_p w_p E_p conj(E_q), w = dOmega A x;
//   - gains, residual, chi^2 partials in FP64 and the adjoint weights (Eq. likelihood);
//   - the pixel adjoint xbar_p = dOmega A sum_{p<q} Re[conj(omega_pq) K_pq];
//   - deterministic reductions (fixed order, no floating-point atomics).
#include <type_traits>

#include "fm_internal.cuh"

namespace fm {

template <typename R> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

// ---------------------------------------------------------------- phasors
// FP32: phase in turns from two-float products so its fractional part keeps ~2^-24
// absolute accuracy even at 60 turns; every product and sum of the error-free
// transformations is explicitly rounded (no contraction into FMAs).
__device__ __forceinline__ float phase_frac_2f(const float *__restrict__ kap, const float *__restrict__ s)
{
    float accf = 0.f, acce = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float kh = kap[2 * c], kl = kap[2 * c + 1], sh = s[2 * c], sl = s[2 * c + 1];
        float p = __fmul_rn(kh, sh);
        float e = __fmaf_rn(kh, sh, -p);                 // exact rounding error of p
        float f = __fsub_rn(p, rintf(p));                // exact: p minus its nearest integer
        accf = __fadd_rn(accf, f);
        acce = __fadd_rn(acce, __fadd_rn(e, __fmaf_rn(kh, sl, __fmul_rn(kl, sh))));
    }
    float t = __fadd_rn(accf, acce);
    return __fsub_rn(t, rintf(t));
}

template <typename R> struct Phasor;
template <> struct Phasor<float> {
    static __device__ __forceinline__ void eval(const DevGeom &g, int f, int i, int t, int p, float &re, float &im)
    {
        float fr = phase_frac_2f(g.kap32 + ((size_t)f * g.A + i) * 6, g.s32 + ((size_t)t * g.npix + p) * 6);
        float sn, cs;
        sincospif(2.0f * fr, &sn, &cs);
        re = cs;
        im = -sn;
    }
};
template <> struct Phasor<double> {
    static __device__ __forceinline__ void eval(const DevGeom &g, int f, int i, int t, int p, double &re, double &im)
    {
        const double *k = g.kap64 + ((size_t)f * g.A + i) * 3;
        const double *s = g.s64 + ((size_t)t * g.npix + p) * 3;
        double ph = k[0] * s[0] + k[1] * s[1] + k[2] * s[2];
        ph -= rint(ph);
        double sn, cs;
        sincospi(2.0 * ph, &sn, &cs);
        re = cs;
        im = -sn;
    }
};

// Beam-weighted solid angle dOmega_d A(za; nu) of pixel p at LST t.
// (Gaussian beam from the squared zenith angle; the Airy beam from its table)
template <typename R>
__device__ __forceinline__ R pixel_weight(const DevGeom &g, int f, int t, int p)
{
    if (g.beam64) return Tab<R>::domega(g)[p / g.R] * (R)g.beam64[((size_t)f * g.T + t) * g.npix + p];
    R z2 = Tab<R>::za2(g)[(size_t)t * g.npix + p];
    if (z2 < R(0)) return R(0);
    return Tab<R>::domega(g)[p / g.R] * exp(Tab<R>::bcoef(g)[f] * z2);
}
template <>
__device__ __forceinline__ float pixel_weight<float>(const DevGeom &g, int f, int t, int p)
{
    if (g.beam32) return g.domega32[p / g.R] * g.beam32[((size_t)f * g.T + t) * g.npix + p];
    float z2 = g.za2_32[(size_t)t * g.npix + p];
    if (z2 < 0.f) return 0.f;
    return g.domega32[p / g.R] * __expf(g.bcoef32[f] * z2);
}

__host__ __device__ __forceinline__ int pair_index(int i, int j, int A)
{
    return i * A - (i * (i + 1)) / 2 + (j - i - 1);
}

// ---------------------------------------------------------------- GEMM
struct GemmArgs {
    int M, N, K;
    long long sAb, sAi, sAk, sBb, sBk, sBj, sCb, sCi, sCj;
    int zero_b00;      // read B[0][0] of every batch as zero (drops the monopole mode a_00)
};

template <typename R>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs a, const R *__restrict__ A, const R *__restrict__ B,
                                              R *__restrict__ C)
{
    __shared__ R sA[16][65];
    __shared__ R sB[16][65];
    const int b = blockIdx.z, i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
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
            sB[kb][jj] = (gj < a.N && gk2 < a.K && !(a.zero_b00 && gj == 0 && gk2 == 0)) ? Bb[gk2 * a.sBk + gj * a.sBj]
                                                                                          : R(0);
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
static fm_status gemm(const GemmArgs &a, int batch, const R *A, const R *B, R *C, cudaStream_t st)
{
    dim3 grid(cdiv(a.N, 64), cdiv(a.M, 64), batch);
    k_gemm<R><<<grid, 256, 0, st>>>(a, A, B, C);
    FM_CK_LAUNCH();
    return FM_OK;
}

template <typename R> static const R *tab_phi(const Ctx &c);
template <> const double *tab_phi<double>(const Ctx &c) { return c.g.phi64; }
template <> const float *tab_phi<float>(const Ctx &c) { return c.g.phi32; }
template <typename R> static const R *tab_leg(const Ctx &c);
template <> const double *tab_leg<double>(const Ctx &c) { return c.g.leg64; }
template <> const float *tab_leg<float>(const Ctx &c) { return c.g.leg32; }

// x[f][d][r] = sum_n P[d][n] sum_m Phi[r][m] a[f][m][n]   (Eq. fg_separable)
template <typename R>
fm_status launch_modes_forward(Ctx &c, const R *a, R *x, cudaStream_t st, int skip_dc, unsigned *xmax,
                               const StripArgs *strips)
{
    if constexpr (std::is_same<R, float>::value)
        if (c.mtc.on) return launch_modes_tc_forward(c, a, x, st, skip_dc, xmax, strips);
    if (xmax || strips) {
        set_error("channel maxima are formed only by the tensor-core mode transform");
        return FM_ERR_STATE;
    }
    R *t1 = (R *)c.tmp;
    GemmArgs s1{c.R, c.N, c.M, 0, c.M, 1, c.nk, c.N, 1, (long long)c.R * c.N, c.N, 1, skip_dc};
    FM_TRY(gemm<R>(s1, c.F, tab_phi<R>(c), a, t1, st));
    GemmArgs s2{c.D, c.R, c.N, 0, c.N, 1, (long long)c.R * c.N, 1, c.N, c.npix, c.R, 1, 0};
    return gemm<R>(s2, c.F, tab_leg<R>(c), t1, x, st);
}

// abar[f][m][n] = sum_r Phi[r][m] sum_d xbar[f][d][r] P[d][n]   (transpose of the above)
template <typename R>
fm_status launch_modes_adjoint(Ctx &c, const R *xbar, R *abar, cudaStream_t st)
{
    if constexpr (std::is_same<R, float>::value)
        if (c.mtc.on) return launch_modes_tc_adjoint(c, xbar, abar, st);
    R *t2 = (R *)c.tmp;
    GemmArgs s1{c.R, c.N, c.D, c.npix, 1, c.R, 0, c.N, 1, (long long)c.R * c.N, c.N, 1, 0};
    FM_TRY(gemm<R>(s1, c.F, xbar, tab_leg<R>(c), t2, st));
    GemmArgs s2{c.M, c.N, c.R, 0, 1, c.M, (long long)c.R * c.N, c.N, 1, c.nk, c.N, 1, 0};
    return gemm<R>(s2, c.F, tab_phi<R>(c), t2, abar, st);
}

// ---------------------------------------------------------------- gains
template <typename R>
__global__ void k_gains(DevGeom g, const R *__restrict__ gamma, R *__restrict__ out)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.F * g.A) return;
    int f = e / g.A, i = e % g.A;
    const R *X = Tab<R>::gleg(g) + (size_t)f * g.NG;
    R re = 0, im = 0;
    for (int k = 0; k < g.NG; ++k) {
        re += X[k] * gamma[(i * g.NG + k) * 2];
        im += X[k] * gamma[(i * g.NG + k) * 2 + 1];
    }
    out[2 * e] = re;
    out[2 * e + 1] = im;
}

template <typename R>
fm_status launch_gains(Ctx &c, const R *gamma, R *g, cudaStream_t st)
{
    k_gains<R><<<cdiv(c.F * c.A, 128), 128, 0, st>>>(c.g, gamma, g);
    FM_CK_LAUNCH();
    return FM_OK;
}

// m_pq = g_p conj(g_q) V_pq
template <typename R>
__global__ void k_apply_gains(DevGeom g, const R *__restrict__ vis, const R *__restrict__ gains, R *__restrict__ out)
{
    long long n = (long long)g.F * g.T * g.B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int b = (int)(e % g.B);
        int f = (int)(e / ((long long)g.T * g.B));
        int i = g.bl_i[b], j = g.bl_j[b];
        R gir = gains[2 * (f * g.A + i)], gii = gains[2 * (f * g.A + i) + 1];
        R gjr = gains[2 * (f * g.A + j)], gji = gains[2 * (f * g.A + j) + 1];
        R ggr = gir * gjr + gii * gji, ggi = gii * gjr - gir * gji;   // g_i conj(g_j)
        R vr = vis[2 * e], vi = vis[2 * e + 1];
        out[2 * e] = ggr * vr - ggi * vi;
        out[2 * e + 1] = ggr * vi + ggi * vr;
    }
}

template <typename R>
fm_status launch_apply_gains(Ctx &c, const R *vis, const R *g, R *out, cudaStream_t st)
{
    k_apply_gains<R><<<1024, 256, 0, st>>>(c.g, vis, g, out);
    FM_CK_LAUNCH();
    return FM_OK;
}

// ---------------------------------------------------------------- forward contraction
// One CTA per (channel, LST).  Pixels stream through shared memory in chunks of PC:
// E and w E are generated there, then each thread accumulates 4x4 antenna tiles
// (p-block <= q-block) of sum_p (w E_p) conj(E_q).  Threads are split into pixel
// groups whose partial sums are added in a fixed order at the end.
template <typename R, int TPT>
__global__ void __launch_bounds__(256) k_vis_simt(DevGeom g, const R *__restrict__ x, R *__restrict__ vis, int nbk,
                                                  int ntile, int tpg, int ngrp, int pc)
{
    using C2 = typename V2<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sEw = reinterpret_cast<C2 *>(smem_raw);
    C2 *sE = sEw + (size_t)pc * g.apad;
    const int ft = blockIdx.x, f = ft / g.T, t = ft % g.T;
    const int tid = threadIdx.x, grp = tid / tpg, lane = tid % tpg;
    int tbi[TPT], tbj[TPT];
    bool tact[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        int tile = lane + k * tpg;
        tact[k] = (grp < ngrp) && (tile < ntile);
        int bi = 0, off = 0;
        if (tact[k]) {
            while (off + (nbk - bi) <= tile) { off += nbk - bi; ++bi; }
        }
        tbi[k] = bi;
        tbj[k] = bi + (tile - off);
    }
    R acc[TPT][4][4][2];
#pragma unroll
    for (int k = 0; k < TPT; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[k][u][v][0] = acc[k][u][v][1] = R(0);

    const R *xf = x + (size_t)f * g.npix;
    R *sW = reinterpret_cast<R *>(sE + (size_t)pc * g.apad);       // [pc]
    for (int p0 = 0; p0 < g.npix; p0 += pc) {
        __syncthreads();
        for (int pl = tid; pl < pc; pl += blockDim.x) {
            int p = p0 + pl;
            sW[pl] = (p < g.npix) ? pixel_weight<R>(g, f, t, p) * xf[p] : R(0);
        }
        __syncthreads();
        for (int e = tid; e < pc * g.apad; e += blockDim.x) {
            int pl = e / g.apad, i = e % g.apad, p = p0 + pl;
            C2 ev, ew;
            ev.x = ev.y = ew.x = ew.y = R(0);
            if (i < g.A && p < g.npix) {
                R w = sW[pl];
                R er, ei;
                Phasor<R>::eval(g, f, i, t, p, er, ei);
                ev.x = er; ev.y = ei;
                ew.x = w * er; ew.y = w * ei;
            }
            sE[e] = ev;
            sEw[e] = ew;
        }
        __syncthreads();
        if (grp < ngrp) {
            // chunk partial sums first, then one add into the running total: the
            // rounding error grows with pc/ngrp + npix/pc terms instead of npix/ngrp
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (!tact[k]) continue;
                R part[4][4][2];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) part[u][v][0] = part[u][v][1] = R(0);
                for (int pl = grp; pl < pc; pl += ngrp) {
                    const C2 *rw = sEw + (size_t)pl * g.apad;
                    const C2 *rv = sE + (size_t)pl * g.apad;
                    C2 av[4], bv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) { av[q] = rw[4 * tbi[k] + q]; bv[q] = rv[4 * tbj[k] + q]; }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            part[u][v][0] += av[u].x * bv[v].x + av[u].y * bv[v].y;
                            part[u][v][1] += av[u].y * bv[v].x - av[u].x * bv[v].y;
                        }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        acc[k][u][v][0] += part[u][v][0];
                        acc[k][u][v][1] += part[u][v][1];
                    }
            }
        }
    }
    __syncthreads();
    R *red = reinterpret_cast<R *>(smem_raw);       // [ngrp][ntile][16][2]
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        if (!tact[k]) continue;
        int tile = lane + k * tpg;
        R *dst = red + ((size_t)grp * ntile + tile) * 32;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                dst[(u * 4 + v) * 2] = acc[k][u][v][0];
                dst[(u * 4 + v) * 2 + 1] = acc[k][u][v][1];
            }
    }
    __syncthreads();
    for (int e = tid; e < ntile * 16; e += blockDim.x) {
        int tile = e / 16, q = e % 16, u = q / 4, v = q % 4;
        int bi = 0, off = 0;
        while (off + (nbk - bi) <= tile) { off += nbk - bi; ++bi; }
        int bj = bi + (tile - off);
        int i = 4 * bi + u, j = 4 * bj + v;
        if (i < j && j < g.A) {
            R re = 0, im = 0;
            for (int gq = 0; gq < ngrp; ++gq) {
                re += red[((size_t)gq * ntile + tile) * 32 + 2 * q];
                im += red[((size_t)gq * ntile + tile) * 32 + 2 * q + 1];
            }
            size_t o = ((size_t)ft * g.B + pair_index(i, j, g.A)) * 2;
            vis[o] = re;
            vis[o + 1] = im;
        }
    }
}

template <typename R, int TPT>
static fm_status vis_simt_launch(Ctx &c, const R *x, R *vis, cudaStream_t st)
{
    int nbk = (c.A + 3) / 4, ntile = nbk * (nbk + 1) / 2;
    int tpg = ((cdiv(ntile, TPT) + 31) / 32) * 32;
    if (tpg > 256) { set_error("direct forward: %d antennas exceed the tile layout", c.A); return FM_ERR_UNSUPPORTED; }
    int ngrp = 256 / tpg;
    // pixels staged per round: 64, halved while the phasor tiles exceed shared memory
    int pc = 64;
    size_t sm_e = 0, smem = 0;
    const size_t sm_r = (size_t)ngrp * ntile * 32 * sizeof(R);
    for (;; pc /= 2) {
        sm_e = 2 * (size_t)pc * c.g.apad * 2 * sizeof(R) + pc * sizeof(R);
        smem = sm_e > sm_r ? sm_e : sm_r;
        if (smem <= 227 * 1024 || pc <= 8) break;
    }
    if (smem > 227 * 1024) { set_error("direct forward: tiles exceed shared memory"); return FM_ERR_UNSUPPORTED; }
    FM_CK(smem_opt_in(k_vis_simt<R, TPT>));
    k_vis_simt<R, TPT><<<c.F * c.T, 256, smem, st>>>(c.g, x, vis, nbk, ntile, tpg, ngrp, pc);
    FM_CK_LAUNCH();
    return FM_OK;
}

template <typename R>
fm_status launch_vis(Ctx &c, const R *x, R *vis, cudaStream_t st)
{
    int nbk = (c.A + 3) / 4, ntile = nbk * (nbk + 1) / 2;
    if (ntile <= 256) return vis_simt_launch<R, 1>(c, x, vis, st);
    if (ntile <= 512) return vis_simt_launch<R, 2>(c, x, vis, st);
    if (ntile <= 1024) return vis_simt_launch<R, 4>(c, x, vis, st);
    return vis_simt_launch<R, 8>(c, x, vis, st);
}

// ---------------------------------------------------------------- chi^2 epilogue
template <typename R>
__device__ void block_sum_double(double v, double *out, double *sred)
{
    sred[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sred[threadIdx.x] += sred[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sred[0];
}

// One CTA per (channel, LST): model, residual, chi^2 partial (FP64), the adjoint
// weights omega_pq = conj(g_p) g_q r_pq / sigma^2 and the per-antenna gain-gradient
// partials Z_a (gradient w.r.t. gamma_ak is X_k(nu) (Re Z_a, Im Z_a)).
template <typename R>
__global__ void __launch_bounds__(256) k_chi2_mid(DevGeom g, const R *__restrict__ vis, const R *__restrict__ data,
                                                  const R *__restrict__ gains, R *__restrict__ omega,
                                                  R *__restrict__ zpart, double *__restrict__ chi2p)
{
    using C2 = typename V2<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sred = reinterpret_cast<double *>(smem_raw);            // [256]
    C2 *sG = reinterpret_cast<C2 *>(sred + 256);                      // [A]
    C2 *sV = sG + g.A;                                                // [B]
    C2 *sRr = sV + g.B;                                               // [B]
    const int ft = blockIdx.x, f = ft / g.T;
    for (int i = threadIdx.x; i < g.A; i += blockDim.x) {
        sG[i].x = gains[2 * (f * g.A + i)];
        sG[i].y = gains[2 * (f * g.A + i) + 1];
    }
    __syncthreads();
    const R is2 = (R)g.inv_sigma2;
    double c2 = 0.0;
    for (int b = threadIdx.x; b < g.B; b += blockDim.x) {
        int i = g.bl_i[b], j = g.bl_j[b];
        size_t o = ((size_t)ft * g.B + b) * 2;
        C2 V, gi = sG[i], gj = sG[j];
        V.x = vis[o]; V.y = vis[o + 1];
        R ggr = gi.x * gj.x + gi.y * gj.y, ggi = gi.y * gj.x - gi.x * gj.y;     // g_i conj(g_j)
        R rr = ggr * V.x - ggi * V.y - data[o];
        R ri = ggr * V.y + ggi * V.x - data[o + 1];
        c2 += (double)rr * (double)rr + (double)ri * (double)ri;
        // omega = conj(g_i) g_j r / sigma^2 = conj(g_i conj(g_j)) r / sigma^2
        omega[o] = (ggr * rr + ggi * ri) * is2;
        omega[o + 1] = (ggr * ri - ggi * rr) * is2;
        sV[b] = V;
        sRr[b].x = rr; sRr[b].y = ri;
    }
    block_sum_double<R>(c2, chi2p + ft, sred);
    if (threadIdx.x == 0) chi2p[ft] *= g.inv_sigma2;
    __syncthreads();
    for (int a = threadIdx.x; a < g.A; a += blockDim.x) {
        R zr = 0, zi = 0;
        for (int j = 0; j < g.A; ++j) {
            if (j == a) continue;
            if (j > a) {   // pair (a, j): t = conj(r) conj(g_j) V; Z += conj(t)
                int b = pair_index(a, j, g.A);
                C2 r = sRr[b], V = sV[b], gj = sG[j];
                R cr = r.x * gj.x - r.y * gj.y, ci = -(r.x * gj.y + r.y * gj.x);   // conj(r) conj(g_j)
                R tr = cr * V.x - ci * V.y, ti = cr * V.y + ci * V.x;
                zr += tr; zi -= ti;
            } else {       // pair (j, a): t = conj(r) g_j V; Z += t
                int b = pair_index(j, a, g.A);
                C2 r = sRr[b], V = sV[b], gj = sG[j];
                R cr = r.x * gj.x + r.y * gj.y, ci = r.x * gj.y - r.y * gj.x;      // conj(r) g_j
                zr += cr * V.x - ci * V.y;
                zi += cr * V.y + ci * V.x;
            }
        }
        zpart[((size_t)ft * g.A + a) * 2] = zr * is2;
        zpart[((size_t)ft * g.A + a) * 2 + 1] = zi * is2;
    }
}

// One CTA per (channel, LST): model, residual, chi^2 partial (a warp's terms summed in the
// working type, the warps' sums in FP64), the adjoint weights
// omega_pq = conj(g_p) g_q r_pq / sigma^2 and the per-antenna gain partials
// Z_a = [sum_{q>a} r_aq g_q conj(V_aq) + sum_{p<a} conj(r_pa) g_p V_pa] / sigma^2.  The two
// terms of every baseline are formed once, with its residual; Z_a then sums its A - 1 terms
// in CF_THREADS / A interleaved chunks (one thread each) and adds the chunks in order.  The
// gains g_i(nu_f) = sum_k X_k(nu_f) gamma_ik are formed from the coefficients gamma in the
// prologue.  With q32 != NULL (hour-angle form) omega is not written: its sums over the
// baseline groups go to q32[f][t][u] and their largest |Re|, |Im| to qmax_ft[f][t].  With
// hv.vpart != NULL (hour-angle form, one LST pass) V is formed here from the forward's partial
// sums and the groups' monopole visibilities (HaVSrc) instead of being read from vis.  Needs
// A <= CF_THREADS.
constexpr int CF_THREADS = 256;
template <typename R>
__global__ void __launch_bounds__(CF_THREADS, sizeof(R) == 4 ? 8 : 1) k_chi2_ft(DevGeom g, const R *__restrict__ vis, const R *__restrict__ data,
                                                        const R *__restrict__ gamma, R *__restrict__ omega,
                                                        R *__restrict__ zpart, double *__restrict__ chi2p, int U,
                                                        const int *__restrict__ moff, const int *__restrict__ mem,
                                                        float *__restrict__ q32, float *__restrict__ qmax_ft,
                                                        const R *__restrict__ rin, HaVSrc hv)
{
    using C2 = typename V2<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sG = reinterpret_cast<C2 *>(smem_raw);            // [A]
    C2 *sTi = sG + g.A;                                    // [B] term of baseline (i, j) in Z_i
    C2 *sTj = sTi + g.B;                                   // [B] term of baseline (i, j) in Z_j
    C2 *sW = sTj + g.B;                                    // [B] omega (hour-angle form)
    float *sS = reinterpret_cast<float *>(sW + g.B);       // [nmt][128] forward partial sums (hv)
    __shared__ C2 sZ[CF_THREADS];                          // chunk sums of Z_a
    __shared__ double dred[CF_THREADS / 32];
    __shared__ float fred[CF_THREADS / 32];
    const int ft = blockIdx.x, f = ft / g.T, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    {
        const R *X = Tab<R>::gleg(g) + (size_t)f * g.NG;
        for (int i = tid; i < g.A; i += CF_THREADS) {     // as k_gains
            R re = 0, im = 0;
            for (int k = 0; k < g.NG; ++k) {
                re += X[k] * gamma[(i * g.NG + k) * 2];
                im += X[k] * gamma[(i * g.NG + k) * 2 + 1];
            }
            sG[i].x = re;
            sG[i].y = im;
        }
    }
    float hsc = 0.f, hcf = 0.f;
    if (hv.vpart) {     // the partial rows of every M-tile at this LST, summed in rank order
        const int t = ft - f * g.T;
        for (int e = tid; e < hv.nmt * 128; e += CF_THREADS) {
            const int seg = (e >> 7) * hv.F + f, row = e & 127, nc = hv.ncontrib[seg];
            // the contributors' rows in rank order, four loads ahead
            const float *src = hv.vpart + ((size_t)seg * hv.J * hv.npad + t) * 128 + row;
            const size_t js = (size_t)hv.npad * 128;
            float a = 0.f;
            for (int j0 = 0; j0 < nc; j0 += 4) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = j0 + u < nc ? src[(size_t)(j0 + u) * js] : 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j0 + u < nc) a += v[u];
            }
            sS[e] = a;
        }
        const float mx = __uint_as_float(hv.xmax[f]);
        float s2 = 1.f;
        if (mx > 0.f && isfinite(mx)) {
            int ex;
            frexpf(mx, &ex);
            s2 = ldexpf(1.f, 14 - ex);
        }
        hsc = 1.f / (hv.sp * s2);
        hcf = hv.dc ? hv.dc[(size_t)f * hv.dcs] : 0.f;
    }
    __syncthreads();
    const R is2 = (R)g.inv_sigma2;
    const C2 *vrow = vis ? reinterpret_cast<const C2 *>(vis) + (size_t)ft * g.B : nullptr;
    const C2 *drow = reinterpret_cast<const C2 *>(data) + (size_t)ft * g.B;
    // rin != NULL (delay filter): the residual weights come in precomputed, sigma^2 F^T W F r
    const C2 *rrow = rin ? reinterpret_cast<const C2 *>(rin) + (size_t)ft * g.B : nullptr;
    C2 *orow = reinterpret_cast<C2 *>(omega) + (size_t)ft * g.B;
    R c2 = 0;   // a warp's terms in the working type; FP64 across warps
    for (int b = tid; b < g.B; b += CF_THREADS) {
        const int i = g.bl_i[b], j = g.bl_j[b];
        C2 V;
        if (hv.vpart) {
            const int code = hv.bmap[b], u = code >> 1, row = 128 * (u >> 6) + 2 * (u & 63);
            const float sgn = (code & 1) ? -1.f : 1.f;
            // the roundings of k_ha_vfinish, so that V equals the finished forward's bitwise
            float vx = __fmul_rn(sS[row], hsc), vy = __fmul_rn(sgn * sS[row + 1], hsc);
            if (hv.dc) {
                const float2 u2 = reinterpret_cast<const float2 *>(hv.ug)[(size_t)ft * U + u];
                vx = __fmaf_rn(hcf, u2.x, vx);
                vy = __fmaf_rn(hcf, sgn * u2.y, vy);
            }
            V.x = (R)vx;
            V.y = (R)vy;
        } else {
            V = vrow[b];
        }
        const C2 d = drow[b], gi = sG[i], gj = sG[j];
        const R ggr = gi.x * gj.x + gi.y * gj.y, ggi = gi.y * gj.x - gi.x * gj.y;     // g_i conj(g_j)
        C2 r, om, ti, tj;
        if (rrow) {
            r = rrow[b];
        } else {
            r.x = ggr * V.x - ggi * V.y - d.x;
            r.y = ggr * V.y + ggi * V.x - d.y;
        }
        c2 += r.x * r.x + r.y * r.y;
        om.x = (ggr * r.x + ggi * r.y) * is2;
        om.y = (ggr * r.y - ggi * r.x) * is2;
        if (q32) sW[b] = om;
        else orow[b] = om;
        {   // r g_j conj(V), the term in Z_i
            const R pr = r.x * gj.x - r.y * gj.y, pi = r.x * gj.y + r.y * gj.x;
            ti.x = pr * V.x + pi * V.y;
            ti.y = pi * V.x - pr * V.y;
        }
        {   // conj(r) g_i V, the term in Z_j
            const R pr = r.x * gi.x + r.y * gi.y, pi = r.x * gi.y - r.y * gi.x;
            tj.x = pr * V.x - pi * V.y;
            tj.y = pr * V.y + pi * V.x;
        }
        sTi[b] = ti;
        sTj[b] = tj;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    if (lane == 0) dred[w] = (double)c2;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < CF_THREADS / 32; ++k) a += dred[k];
        chi2p[ft] = a * g.inv_sigma2;
    }
    if (q32) {
        float qm = 0.f;
        for (int u = tid; u < U; u += CF_THREADS) {
            float qr = 0.f, qi = 0.f;
            for (int m = moff[u]; m < moff[u + 1]; ++m) {
                const int code = mem[m], b = code >> 1;
                qr += (float)sW[b].x;
                qi += (code & 1) ? -(float)sW[b].y : (float)sW[b].y;
            }
            float *qo = q32 + ((size_t)ft * U + u) * 2;
            qo[0] = qr;
            qo[1] = qi;
            qm = fmaxf(qm, fmaxf(fabsf(qr), fabsf(qi)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qm = fmaxf(qm, __shfl_xor_sync(0xffffffffu, qm, o));
        if (lane == 0) fred[w] = qm;
    }
    // Z_a, chunk c: partners j = c, c + nc, ... (j != a); pair_index(a, j) = rowa + j for j > a
    const int nc = CF_THREADS / g.A;
    if (tid < nc * g.A) {
        const int a = tid / nc, c = tid - a * nc;
        const int rowa = a * g.A - (a * (a + 1)) / 2 - a - 1;
        R zr = 0, zi = 0;
        for (int j = c; j < g.A; j += nc) {
            if (j == a) continue;
            const C2 t = j > a ? sTi[rowa + j] : sTj[pair_index(j, a, g.A)];
            zr += t.x;
            zi += t.y;
        }
        sZ[tid].x = zr;
        sZ[tid].y = zi;
    }
    __syncthreads();
    if (q32 && tid == 0) {
        float m = 0.f;
        for (int k = 0; k < CF_THREADS / 32; ++k) m = fmaxf(m, fred[k]);
        qmax_ft[ft] = m;
    }
    if (tid < g.A) {
        R zr = 0, zi = 0;
        for (int c = 0; c < nc; ++c) {
            zr += sZ[tid * nc + c].x;
            zi += sZ[tid * nc + c].y;
        }
        zpart[((size_t)ft * g.A + tid) * 2] = zr * is2;
        zpart[((size_t)ft * g.A + tid) * 2 + 1] = zi * is2;
    }
}

// grad_gamma[a][k][c] = sum_{f,t} X_k(nu_f) zpart[f][t][a][c]: one CTA per (a, c); thread
// j takes the (channel, LST) pairs j, j + GR_THREADS, ... in batches of GR_U independent
// loads.  Per thread and across a warp (fixed shuffle order) the sums are in the working
// type; the warps' sums are added in order in FP64 (the FP64 pipe is narrow on this part,
// so it is kept off the per-element path).
constexpr int GR_NGMAX = 8, GR_THREADS = 1024, GR_U = 4;
template <typename R>
__global__ void __launch_bounds__(GR_THREADS) k_gain_reduce_ft(DevGeom g, const R *__restrict__ zpart,
                                                               R *__restrict__ out)
{
    __shared__ double red[GR_THREADS / 32][GR_NGMAX];
    const int a = blockIdx.x >> 1, c = blockIdx.x & 1, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const R *gl = Tab<R>::gleg(g);
    R acc[GR_NGMAX];
#pragma unroll
    for (int k = 0; k < GR_NGMAX; ++k) acc[k] = 0;
    const int nft = g.F * g.T;
    for (int base = 0; base < nft; base += GR_THREADS * GR_U) {
        R z[GR_U];
        int f[GR_U];
#pragma unroll
        for (int u = 0; u < GR_U; ++u) {
            const int ft = base + u * GR_THREADS + (int)threadIdx.x;
            z[u] = ft < nft ? zpart[((size_t)ft * g.A + a) * 2 + c] : (R)0;
            f[u] = ft < nft ? ft / g.T : 0;
        }
#pragma unroll
        for (int u = 0; u < GR_U; ++u)
#pragma unroll
            for (int k = 0; k < GR_NGMAX; ++k)
                if (k < g.NG) acc[k] += gl[(size_t)f[u] * g.NG + k] * z[u];
    }
#pragma unroll
    for (int k = 0; k < GR_NGMAX; ++k) {
        R v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[w][k] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < g.NG) {
        double t = 0.0;
        for (int k = 0; k < GR_THREADS / 32; ++k) t += red[k][threadIdx.x];
        out[(a * g.NG + threadIdx.x) * 2 + c] = (R)t;
    }
}

template <typename R>
fm_status launch_chi2_chan(Ctx &c, const R *vis, const R *gamma, R *omega, R *zpart, double *chi2p, bool groups,
                           cudaStream_t st, const R *rin, const HaVSrc *hv)
{
    if (hv && (!std::is_same<R, float>::value || !groups || rin)) {
        set_error("V from the forward's partial sums: hour-angle form, FP32, no delay filter");
        return FM_ERR_STATE;
    }
    const size_t smem = (c.A + 3 * (size_t)c.B) * 2 * sizeof(R) + (hv ? sizeof(float) * 128 * (size_t)hv->nmt : 0);
    if (smem > 227 * 1024 || c.A > CF_THREADS) {
        set_error("chi^2 epilogue: %d antennas (at most %d, %zu bytes of shared memory)", c.A, CF_THREADS, smem);
        return FM_ERR_UNSUPPORTED;
    }
    FM_CK(smem_opt_in(k_chi2_ft<R>));
    k_chi2_ft<R><<<c.F * c.T, CF_THREADS, smem, st>>>(c.g, vis, (const R *)c.data, gamma, omega, zpart, chi2p, c.ha.U,
                                                c.ha.moff, c.ha.mem, groups ? c.ha.q32 : nullptr, c.ha.qmax_ft, rin,
                                                hv ? *hv : HaVSrc{});
    FM_CK_LAUNCH();
    return FM_OK;
}

template <typename R>
fm_status launch_gain_reduce_chan(Ctx &c, const R *zpart, R *grad_gain, cudaStream_t st)
{
    if (c.NG > GR_NGMAX) return launch_gain_reduce<R>(c, zpart, grad_gain, st);
    k_gain_reduce_ft<R><<<2 * c.A, GR_THREADS, 0, st>>>(c.g, zpart, grad_gain);
    FM_CK_LAUNCH();
    return FM_OK;
}

template <typename R>
fm_status launch_chi2_mid(Ctx &c, const R *vis, const R *g, R *omega, R *zpart, double *chi2p, cudaStream_t st)
{
    size_t smem = 256 * sizeof(double) + (c.A + 2 * (size_t)c.B) * 2 * sizeof(R);
    if (smem > 227 * 1024) return FM_ERR_UNSUPPORTED;
    FM_CK(smem_opt_in(k_chi2_mid<R>));
    k_chi2_mid<R><<<c.F * c.T, 256, smem, st>>>(c.g, vis, (const R *)c.data, g, omega, zpart, chi2p);
    FM_CK_LAUNCH();
    return FM_OK;
}

// Tangent of the epilogue for Hessian-vector products.  With dm = dg_p conj(g_q) V +
// g_p conj(dg_q) V + g_p conj(g_q) dV (JVP), the adjoint weights become
// omega' = [dm conj(g_p) g_q + full * r (conj(dg_p) g_q + conj(g_p) dg_q)] / sigma^2 and
// the gain partials follow the same pattern (full = 0 keeps only the dm terms: GN).
template <typename R>
__global__ void __launch_bounds__(256) k_hvp_mid(DevGeom g, const R *__restrict__ vis, const R *__restrict__ dvis,
                                                 const R *__restrict__ data, const R *__restrict__ gains,
                                                 const R *__restrict__ dgains, int full, R *__restrict__ omega,
                                                 R *__restrict__ zpart)
{
    using C2 = typename V2<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sG = reinterpret_cast<C2 *>(smem_raw);
    C2 *sD = sG + g.A;
    C2 *sV = sD + g.A;
    C2 *sdV = sV + g.B;
    C2 *sRr = sdV + g.B;
    C2 *sdM = sRr + g.B;
    const int ft = blockIdx.x, f = ft / g.T;
    for (int i = threadIdx.x; i < g.A; i += blockDim.x) {
        sG[i].x = gains[2 * (f * g.A + i)];
        sG[i].y = gains[2 * (f * g.A + i) + 1];
        sD[i].x = dgains[2 * (f * g.A + i)];
        sD[i].y = dgains[2 * (f * g.A + i) + 1];
    }
    __syncthreads();
    const R is2 = (R)g.inv_sigma2;
    auto mul = [](C2 a, C2 b) { C2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r; };
    auto cj = [](C2 a) { a.y = -a.y; return a; };
    auto add = [](C2 a, C2 b) { a.x += b.x; a.y += b.y; return a; };
    for (int b = threadIdx.x; b < g.B; b += blockDim.x) {
        int i = g.bl_i[b], j = g.bl_j[b];
        size_t o = ((size_t)ft * g.B + b) * 2;
        C2 V, dV, gi = sG[i], gj = sG[j], di = sD[i], dj = sD[j];
        V.x = vis[o]; V.y = vis[o + 1];
        dV.x = dvis[o]; dV.y = dvis[o + 1];
        C2 gg = mul(gi, cj(gj));
        C2 r = mul(gg, V);
        r.x -= data[o]; r.y -= data[o + 1];
        C2 dm = add(add(mul(mul(di, cj(gj)), V), mul(mul(gi, cj(dj)), V)), mul(gg, dV));
        C2 w = mul(dm, cj(gg));
        if (full) w = add(w, mul(r, add(mul(cj(di), gj), mul(cj(gi), dj))));
        omega[o] = w.x * is2;
        omega[o + 1] = w.y * is2;
        sV[b] = V; sdV[b] = dV; sRr[b] = r; sdM[b] = dm;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < g.A; a += blockDim.x) {
        C2 z;
        z.x = z.y = R(0);
        for (int j = 0; j < g.A; ++j) {
            if (j == a) continue;
            if (j > a) {       // pair (a, j): c = conj(dm) conj(g_j) V + full conj(r)(conj(dg_j) V + conj(g_j) dV)
                int b = pair_index(a, j, g.A);
                C2 c = mul(mul(cj(sdM[b]), cj(sG[j])), sV[b]);
                if (full) c = add(c, mul(cj(sRr[b]), add(mul(cj(sD[j]), sV[b]), mul(cj(sG[j]), sdV[b]))));
                z = add(z, cj(c));
            } else {           // pair (j, a): c = conj(dm) g_j V + full conj(r)(dg_j V + g_j dV)
                int b = pair_index(j, a, g.A);
                C2 c = mul(mul(cj(sdM[b]), sG[j]), sV[b]);
                if (full) c = add(c, mul(cj(sRr[b]), add(mul(sD[j], sV[b]), mul(sG[j], sdV[b]))));
                z = add(z, c);
            }
        }
        zpart[((size_t)ft * g.A + a) * 2] = z.x * is2;
        zpart[((size_t)ft * g.A + a) * 2 + 1] = z.y * is2;
    }
}

template <typename R>
fm_status launch_hvp_mid(Ctx &c, const R *vis, const R *dvis, const R *g, const R *dg, int full, R *omega, R *zpart,
                         cudaStream_t st)
{
    size_t smem = (2 * (size_t)c.A + 4 * (size_t)c.B) * 2 * sizeof(R);
    if (smem > 227 * 1024) return FM_ERR_UNSUPPORTED;
    FM_CK(smem_opt_in(k_hvp_mid<R>));
    k_hvp_mid<R><<<c.F * c.T, 256, smem, st>>>(c.g, vis, dvis, (const R *)c.data, g, dg, full, omega, zpart);
    FM_CK_LAUNCH();
    return FM_OK;
}

// ---------------------------------------------------------------- adjoint contraction
// One CTA per (channel, tile of PT pixels), looping over LSTs so xbar accumulates in
// registers without atomics.  For each LST the tile's phasors go to shared memory and
// each thread forms, for its pixel, sum_p Re[E_p conj(Y_p)] with
// Y_p = sum_{q>p} omega_pq E_q  (= sum_{p<q} Re[conj(omega_pq) E_p conj(E_q)]).
template <typename R>
__global__ void __launch_bounds__(128) k_adj_simt(DevGeom g, const R *__restrict__ omega, R *__restrict__ xbar)
{
    using C2 = typename V2<R>::t;
    constexpr int PT = 128;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sE = reinterpret_cast<C2 *>(smem_raw);        // [A][PT]
    C2 *sC = sE + (size_t)g.A * PT;                   // [B]
    const int f = blockIdx.y, p0 = blockIdx.x * PT, tid = threadIdx.x;
    const int p = p0 + tid;
    R accx = R(0);
    for (int t = 0; t < g.T; ++t) {
        __syncthreads();
        for (int e = tid; e < g.A * PT; e += blockDim.x) {
            int i = e / PT, pl = e % PT, pp = p0 + pl;
            C2 ev;
            ev.x = ev.y = R(0);
            if (pp < g.npix) Phasor<R>::eval(g, f, i, t, pp, ev.x, ev.y);
            sE[e] = ev;
        }
        const R *om = omega + ((size_t)(f * g.T + t) * g.B) * 2;
        for (int b = tid; b < g.B; b += blockDim.x) {
            sC[b].x = om[2 * b];
            sC[b].y = om[2 * b + 1];
        }
        __syncthreads();
        if (p < g.npix) {
            R w = pixel_weight<R>(g, f, t, p);
            if (w != R(0)) {
                R acc = R(0);
                for (int i = 0; i + 1 < g.A; ++i) {
                    R yr = 0, yi = 0;
                    int b0 = pair_index(i, i + 1, g.A) - (i + 1);
                    for (int j = i + 1; j < g.A; ++j) {
                        C2 cc = sC[b0 + j], ej = sE[(size_t)j * PT + tid];
                        yr += cc.x * ej.x - cc.y * ej.y;
                        yi += cc.x * ej.y + cc.y * ej.x;
                    }
                    C2 ei = sE[(size_t)i * PT + tid];
                    acc += ei.x * yr + ei.y * yi;
                }
                accx += w * acc;
            }
        }
    }
    if (p < g.npix) xbar[(size_t)f * g.npix + p] = accx;
}

template <typename R>
fm_status launch_adjoint(Ctx &c, const R *omega, R *xbar, cudaStream_t st)
{
    size_t smem = ((size_t)c.A * 128 + c.B) * 2 * sizeof(R);
    if (smem > 227 * 1024) return FM_ERR_UNSUPPORTED;
    FM_CK(smem_opt_in(k_adj_simt<R>));
    dim3 grid(cdiv(c.npix, 128), c.F);
    k_adj_simt<R><<<grid, 128, smem, st>>>(c.g, omega, xbar);
    FM_CK_LAUNCH();
    return FM_OK;
}

// ---------------------------------------------------------------- reductions
// grad_gamma[a][k][re, im] = sum_{f,t} X_k(nu_f) Z[f][t][a]   (FP64, fixed order)
template <typename R>
__global__ void __launch_bounds__(256) k_gain_reduce(DevGeom g, const R *__restrict__ zpart, R *__restrict__ out)
{
    __shared__ double sred[256];
    const int a = blockIdx.x, k = blockIdx.y;
    double sr = 0.0, si = 0.0;
    for (int ft = threadIdx.x; ft < g.F * g.T; ft += blockDim.x) {
        int f = ft / g.T;
        double X = (double)Tab<R>::gleg(g)[(size_t)f * g.NG + k];
        sr += X * (double)zpart[((size_t)ft * g.A + a) * 2];
        si += X * (double)zpart[((size_t)ft * g.A + a) * 2 + 1];
    }
    double tot;
    block_sum_double<R>(sr, &tot, sred);
    __syncthreads();
    if (threadIdx.x == 0) out[(a * g.NG + k) * 2] = (R)tot;
    __syncthreads();
    block_sum_double<R>(si, &tot, sred);
    if (threadIdx.x == 0) out[(a * g.NG + k) * 2 + 1] = (R)tot;
}

template <typename R>
fm_status launch_gain_reduce(Ctx &c, const R *zpart, R *grad_gain, cudaStream_t st)
{
    dim3 grid(c.A, c.NG);
    k_gain_reduce<R><<<grid, 256, 0, st>>>(c.g, zpart, grad_gain);
    FM_CK_LAUNCH();
    return FM_OK;
}

// fixed-order sum over a CTA of 256 threads: lane shuffles in T, then the 8 warps' sums in
// order in FP64; the result is valid in thread 0
template <typename T>
__device__ __forceinline__ double cta256_sum(T v, double *wred)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) t += wred[k];
    __syncthreads();
    return t;
}

template <typename R>
struct __align__(16) Pack16 { R v[16 / sizeof(R)]; };

// grad += lam (theta - mu) and the prior energy sum lam (theta - mu)^2 / 2 (a warp's terms
// summed in the working type, the warps' sums in FP64), then chi^2 = sum of the per-(f,t)
// partials (FP64, loads batched so that their latencies overlap) and U = chi^2 / 2 + prior.
// Each CTA writes its partial; the CTA that takes the last ticket adds the partials in
// index order (so the result does not depend on which CTA that is) and resets the ticket
// for the next launch.  With p != NULL the pass also applies the leapfrog momentum kick
// p -= frac eps grad with the finished gradient (eps = prm[0], read on the device).  vec: the
// arrays are 16-byte aligned.
constexpr int PT_THREADS = 256;
template <typename R>
__global__ void __launch_bounds__(PT_THREADS) k_prior_total(long long n, int vec, const R *__restrict__ theta,
                                                            const R *__restrict__ mu, const R *__restrict__ lam,
                                                            R *__restrict__ grad, double *part, int nft,
                                                            const double *__restrict__ chi2p, double *chi2_out,
                                                            double *u_out, int *status, unsigned *ticket,
                                                            R *__restrict__ p, const double *__restrict__ prm,
                                                            double frac)
{
    constexpr int W = 16 / sizeof(R);
    __shared__ double wred[8];
    __shared__ int last;
    const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x, gstride = (long long)gridDim.x * blockDim.x;
    R acc = 0;
    if (lam || p) {
        const R ak = p ? (R)(-frac * prm[0]) : (R)0;      // the kick's factor, as in a separate kick
        long long head = 0;
        if (vec) {
            const long long np = n / W;
            head = np * W;
            const Pack16<R> *th = reinterpret_cast<const Pack16<R> *>(theta);
            const Pack16<R> *mp = reinterpret_cast<const Pack16<R> *>(mu);
            const Pack16<R> *lp = reinterpret_cast<const Pack16<R> *>(lam);
            Pack16<R> *gp = reinterpret_cast<Pack16<R> *>(grad);
            Pack16<R> *pp = reinterpret_cast<Pack16<R> *>(p);
            // two packs a thread at a time (k and k + gstride), all their loads issued first;
            // the terms still go into acc in the order of k
            for (long long k0 = gtid; k0 < np; k0 += 2 * gstride) {
                const long long kk[2] = {k0, k0 + gstride};
                const bool has1 = kk[1] < np;
                Pack16<R> gr[2], t[2], m[2], l[2], pv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (u == 1 && !has1) break;
                    gr[u] = gp[kk[u]];
                    if (lam) {
                        t[u] = th[kk[u]];
                        m[u] = mp[kk[u]];
                        l[u] = lp[kk[u]];
                    }
                    if (p) pv[u] = pp[kk[u]];
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (u == 1 && !has1) break;
                    if (lam) {
#pragma unroll
                        for (int e = 0; e < W; ++e) {
                            const R dv = t[u].v[e] - m[u].v[e], ld = l[u].v[e] * dv;
                            gr[u].v[e] += ld;
                            acc += ld * dv;
                        }
                        gp[kk[u]] = gr[u];
                    }
                    if (p) {
#pragma unroll
                        for (int e = 0; e < W; ++e) pv[u].v[e] += ak * gr[u].v[e];
                        pp[kk[u]] = pv[u];
                    }
                }
            }
        }
        for (long long k = head + gtid; k < n; k += gstride) {
            R gk = grad[k];
            if (lam) {
                const R l = lam[k], dv = theta[k] - mu[k], ld = l * dv;
                gk += ld;
                grad[k] = gk;
                acc += ld * dv;
            }
            if (p) p[k] += ak * gk;
        }
    }
    const double blk = cta256_sum<R>((R)0.5 * acc, wred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = blk;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i0 = 0; i0 < nft; i0 += 8 * PT_THREADS) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * PT_THREADS + (int)threadIdx.x;
            v[u] = i < nft ? __ldcg(chi2p + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) a += v[u];
    }
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) b += __ldcg(part + i);
    const double ta = cta256_sum<double>(a, wred), tb = cta256_sum<double>(b, wred);
    if (threadIdx.x == 0) {
        if (chi2_out) *chi2_out = ta;
        if (u_out) *u_out = 0.5 * ta + tb;
        if (!isfinite(ta) || !isfinite(tb)) atomicExch(status, (int)FM_ERR_NONFINITE);
        *ticket = 0u;
    }
}

template <typename R>
fm_status launch_prior_and_total(Ctx &c, const R *theta, R *grad, const double *chi2p, int nchi2, double *chi2_out,
                                 double *u_out, cudaStream_t st, R *kick_p, const double *kick_prm, double kick_frac)
{
    const R *mu = (const R *)c.mu, *lam = c.have_prior ? (const R *)c.lam : nullptr;
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const int vec = al(theta) && al(mu) && al(c.lam) && al(grad) && al(kick_p);
    const long long units = vec ? c.n_par / (16 / (long long)sizeof(R)) : c.n_par;
    const int nblk = (int)std::max(1LL, std::min<long long>(4 * 152, (long long)cdiv(units, PT_THREADS)));
    k_prior_total<R><<<nblk, PT_THREADS, 0, st>>>(c.n_par, vec, theta, mu, lam, grad, c.red, nchi2, chi2p, chi2_out,
                                                 u_out, c.status, c.ticket, kick_p, kick_prm, kick_frac);
    FM_CK_LAUNCH();
    return FM_OK;
}

template <typename R>
__global__ void k_prior_hvp(long long n, const R *__restrict__ v, const R *__restrict__ lam, R *__restrict__ hv)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        hv[k] += lam[k] * v[k];
}

template <typename R>
fm_status launch_prior_hvp(Ctx &c, const R *v, R *hv, cudaStream_t st)
{
    if (!c.have_prior) return FM_OK;
    k_prior_hvp<R><<<296, 256, 0, st>>>(c.n_par, v, (const R *)c.lam, hv);
    FM_CK_LAUNCH();
    return FM_OK;
}

// ---------------------------------------------------------------- monopole split
// vis[f][t][b] += c_f U[f][t][b] with c_f = src[f * stride]: puts back the visibility of
// the uniform part of the sky that the contraction kernels did not see.
template <typename R>
__global__ void k_add_dc(DevGeom g, const R *__restrict__ src, long long stride, const float *__restrict__ U,
                         R *__restrict__ vis)
{
    long long n = (long long)g.F * g.T * g.B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int f = (int)(e / ((long long)g.T * g.B));
        R cf = src[(long long)f * stride];
        vis[2 * e] += cf * (R)U[2 * e];
        vis[2 * e + 1] += cf * (R)U[2 * e + 1];
    }
}

template <typename R>
fm_status launch_add_dc(Ctx &c, const R *src, long long stride, R *vis, cudaStream_t st)
{
    k_add_dc<R><<<1024, 256, 0, st>>>(c.g, src, stride, c.dc_u, vis);
    FM_CK_LAUNCH();
    return FM_OK;
}

// per-channel mean of x (fixed-order tree) and x' = x - mean
template <typename R>
__global__ void __launch_bounds__(256) k_center(int npix, const R *__restrict__ x, R *__restrict__ xc,
                                                R *__restrict__ mean)
{
    __shared__ double red[256];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) s += (double)x[(size_t)f * npix + p];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const R m = (R)(red[0] / npix);
    if (threadIdx.x == 0) mean[f] = m;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) xc[(size_t)f * npix + p] = x[(size_t)f * npix + p] - m;
}

template <typename R>
fm_status launch_center(Ctx &c, const R *x, R *xc, R *mean, cudaStream_t st)
{
    k_center<R><<<c.F, 256, 0, st>>>(c.npix, x, xc, mean);
    FM_CK_LAUNCH();
    return FM_OK;
}

__global__ void k_d2f(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}

fm_status launch_d2f(long long n, const double *a, float *b, cudaStream_t st)
{
    k_d2f<<<1024, 256, 0, st>>>(n, a, b);
    FM_CK_LAUNCH();
    return FM_OK;
}

#define FM_INST(R)                                                                                       \
    template fm_status launch_chi2_chan<R>(Ctx &, const R *, const R *, R *, R *, double *, bool, cudaStream_t, const R *, \
                                           const HaVSrc *);                                              \
    template fm_status launch_gain_reduce_chan<R>(Ctx &, const R *, R *, cudaStream_t);                 \
    template fm_status launch_modes_forward<R>(Ctx &, const R *, R *, cudaStream_t, int, unsigned *,        \
                                               const StripArgs *);                                           \
    template fm_status launch_modes_adjoint<R>(Ctx &, const R *, R *, cudaStream_t);                     \
    template fm_status launch_gains<R>(Ctx &, const R *, R *, cudaStream_t);                             \
    template fm_status launch_vis<R>(Ctx &, const R *, R *, cudaStream_t);                               \
    template fm_status launch_adjoint<R>(Ctx &, const R *, R *, cudaStream_t);                           \
    template fm_status launch_apply_gains<R>(Ctx &, const R *, const R *, R *, cudaStream_t);            \
    template fm_status launch_chi2_mid<R>(Ctx &, const R *, const R *, R *, R *, double *, cudaStream_t); \
    template fm_status launch_hvp_mid<R>(Ctx &, const R *, const R *, const R *, const R *, int, R *, R *, \
                                         cudaStream_t);                                                  \
    template fm_status launch_gain_reduce<R>(Ctx &, const R *, R *, cudaStream_t);                       \
    template fm_status launch_prior_and_total<R>(Ctx &, const R *, R *, const double *, int, double *, double *, \
                                                 cudaStream_t, R *, const double *, double);             \
    template fm_status launch_prior_hvp<R>(Ctx &, const R *, R *, cudaStream_t);                         \
    template fm_status launch_add_dc<R>(Ctx &, const R *, long long, R *, cudaStream_t);                \
    template fm_status launch_center<R>(Ctx &, const R *, R *, R *, cudaStream_t);
FM_INST(float)
FM_INST(double)

}  // namespace fm
