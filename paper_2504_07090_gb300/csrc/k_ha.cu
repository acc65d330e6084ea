// Hour-angle form of the fringe contraction for drift scans (sm_103a tcgen05).
//
// Eq. (rime_discrete) with K_ij = E_i conj(E_j) sums, for every baseline, channel and
// LST, the beam- and solid-angle-weighted sky times the fringe over all pixels.  In a
// drift scan (Sec. 2.1: the array points at a fixed topocentric direction) with LSTs
// spaced by k / q RA pixels (q <= 4), LST_t - RA_r = LST_0 - RA_{R-1} + (t k - r q + (R - 1) q) dRA / q,
// so the direction of pixel (r, d) at LST t depends on the hour-angle index
// n = t k - r q + (R - 1) q only (cells of dRA / q; q = 1 when the step is a whole number of
// pixels).  With one primary beam for all antennas (Sec. 3.4), baselines
// with equal vectors b = r_i - r_j (up to sign) also have equal (or conjugate) fringes.
// For one channel and one fringe group u the visibility is then
//   V_u(t) = sum_{d, n} P_u(n, d) x((t k + (R - 1) q - n) / q, d)   (terms with q | t k - n),
//   P_u(n, d) = E_i(n, d) conj(E_j(n, d)),  E_i = sqrt(dOmega_d A(n, d)) exp(-2 pi i nu r_i . s(n, d) / c),
// a real GEMM  D[rho][t] = sum_K A[rho][K] B[t][K],  rho = (u, Re | Im), K = (d, n),
// whose A operand is generated tile by tile from a per-channel table of E (computed once
// per handle with FP64 phases) and whose B operand is the Toeplitz matrix of the sky (a
// Hankel matrix once the cells are taken in reverse order), read by the tensor core from
// one shared-memory image per (channel, declination).
//
// The adjoint (the pixel gradient through the same response) is
//   xbar(r, d) = sum_t sum_rho P_rho(n(r, t), d) Q_rho(t),   Q_u = sum_{b in u} omega_b,
// (conj(omega_b) for baselines reversed with respect to the group's representative): the
// GEMM X[n][t] = sum_rho P^T[n][rho] Q[t][rho], then sums along the diagonals
// n = t k + (R - 1 - r) q, done in the epilogue.
//
// Both kernels are warp-specialised: 16 producer warps write the P operand into TMEM,
// one thread issues tcgen05.mma (A from TMEM, B from shared memory) into TMEM
// accumulators, epilogue warps drain them, and single threads issue bulk copies.  LSTs
// beyond 64 run as further passes over the same table.  Every wait is bounded; a timeout
// records FM_ERR_TIMEOUT and the CTA winds down in order.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fm_internal.cuh"
#include "tc_ptx.cuh"

namespace fm {
namespace {

using namespace tc;

// the adjoint's roles (the forward's are the HF_ constants below)
constexpr int HA_PROD_WARPS = 16;
constexpr int HA_EPI_WARP0 = 16;          // warps 16..19 drain TMEM (lane quarter = warp & 3)
constexpr int HA_MMA_WARP = 20;
constexpr int HA_LOAD_WARP = 21;          // bulk copies of the phasor table (and sky strips)
constexpr int HA_QLOAD_WARP = 22;         // adjoint only: bulk copies of the residual tiles
constexpr int HA_EPI2_WARP0 = 23;         // adjoint only: warps 23..26, the second epilogue set
constexpr int HA_ADJ_THREADS = 27 * 32;   // adjoint
constexpr int HA_SUB = 4;                 // 64-cell K chunks per TMEM accumulation chain (shorter chains: less FP32 accumulation bias)
constexpr int HA_SMEM_BUDGET = 227 * 1024 - 1024 - 512;
constexpr int HA_EW = 66;                 // float2 entries per table row: 64 cells + 16 bytes of padding
constexpr int HA_NSTAGE = 4;              // adjoint operand stages (A in TMEM, B in shared memory)
constexpr int HA_TCHUNK = 64;             // LSTs per pass (the GEMM's N); more run as several passes
constexpr int HA_NSTAGE_FWD = 5;          // forward A stages in TMEM
// the forward's roles: HF_PROD_WARPS producer warps in HF_PGROUPS groups of four (one unit each),
// then four TMEM-drain warps, the MMA warp and the bulk-copy warp
constexpr int HF_PROD_WARPS = 12;
constexpr int HF_PGROUPS = HF_PROD_WARPS / 4;
constexpr int HF_EPI_WARP0 = HF_PROD_WARPS;
constexpr int HF_MMA_WARP = HF_PROD_WARPS + 4;
constexpr int HF_LOAD_WARP = HF_PROD_WARPS + 5;
constexpr int HF_THREADS = (HF_PROD_WARPS + 6) * 32;
static_assert((HF_MMA_WARP & 3) == 0 && HF_EPI_WARP0 + 4 == HF_MMA_WARP, "the MMA warp on the first sub-partition");

// kernel parameters, by value
struct HaDev {
    int F, D, T, R, A, U, k, q, nhp, nbc, npad, Ly, Jc, nchunk, nmt, nkq, J;   // k: LST step, q: cells per pixel
    int Tt, t0, Lyc;                      // all LSTs; this LST chunk: [t0, t0 + T); strip bytes / 2 it reads
    long long Q;                          // forward work units: nmt * F * nchunk
    const float2 *E;                      // phasor table, cells paired (forward)
    const float2 *Ea;                     // the same, one (Re, Im) per cell (adjoint)
    const int2 *uij;
};

struct HaLayout {
    int nstage, neslot, ncols, abase, acols;   // TMEM: allocated columns, first A column, columns per A stage
    uint32_t b_bytes, stage_bytes, eslot_bytes, img_bytes;
    uint32_t e_off, v_off, bar_off;
    size_t smem;
};

// 8-byte shared-memory load at a 32-bit shared address
__device__ __forceinline__ float2 lds_f2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// first work unit of CTA g when Q units are cut into G contiguous ranges
__host__ __device__ __forceinline__ long long range_lo(long long Q, int G, int g) { return Q * g / G; }

__host__ __device__ inline int cta_of(long long q, long long Q, int G)
{
    int g = (int)(q * G / Q);
    while (g + 1 < G && range_lo(Q, G, g + 1) <= q) ++g;
    while (g > 0 && range_lo(Q, G, g) > q) --g;
    return g;
}

// power of two putting max below 2^14 (FP16 operand range), 1 for 0 or non-finite
__device__ __forceinline__ float pow2_scale(float mx)
{
    float sc = 1.f;
    if (mx > 0.f && isfinite(mx)) {
        int e;
        frexpf(mx, &e);
        sc = ldexpf(1.f, 14 - e);
    }
    return sc;
}

// ------------------------------------------------------------ per-handle phasor table
// E[f][d][nb][i][row], n = 64 nb + nl, i over the table's antenna subset plus one all-zero
// entry (padding pairs point at it).  A row of 132 floats holds the 64 cells, then 16 bytes
// of padding so that rows of different antennas start in different shared-memory banks;
// `paired` = 1 (forward): the cells in pairs, (Re E_n, Re E_n+1, Im E_n, Im E_n+1) for even
// n (one 16-byte load feeds packed FP32x2 arithmetic on two cells); 0 (adjoint): (Re, Im)
// per cell.  Each cell holds
// sqrt(dOmega_d A(za; nu_f)) 2^(e/2) exp(-2 pi i nu r_i . s / c)
// at hour angle H(n) = LST_0 - (ra_min + (R - 1 - n + 1/2) dRA); zero below the horizon
// and for n >= nh.  FP64 throughout, stored as FP32.
struct HaTabArgs {
    int F, D, R, A, A_all, nh, nhp, nbc, q;
    int ant[64];                          // table entry -> antenna index
    double lst0, ra_min, dra, dec_min, ddec, lat, amp_scale;
    const double *kap64, *bcoef64, *domega64;
    int airy;                             // Airy beam (Eq. airy) instead of the Gaussian
    double dew, dns;
    const double *freq;
};

__global__ void k_ha_table(HaTabArgs a, int paired, float *__restrict__ E)
{
    const long long total = (long long)a.F * a.D * a.nbc * a.A * HA_EW;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int nl = (int)(e % HA_EW);
        long long r = e / HA_EW;
        const int i = (int)(r % a.A);
        r /= a.A;
        const int nb = (int)(r % a.nbc);
        r /= a.nbc;
        const int d = (int)(r % a.D);
        const int f = (int)(r / a.D);
        const int n = 64 * nb + nl;
        float2 out = make_float2(0.f, 0.f);
        if (nl < 64 && n < a.nh && i < a.A - 1) {     // entry A - 1 is the zero antenna of padded pairs
            const double H = a.lst0 - (a.ra_min + ((double)((a.R - 1) * a.q - n) + 0.5 * a.q) * (a.dra / a.q));
            const double dec = a.dec_min + (d + 0.5) * a.ddec;
            double sd, cd, sh, ch, sl, cl;
            sincos(dec, &sd, &cd);
            sincos(H, &sh, &ch);
            sincos(a.lat, &sl, &cl);
            const double sE = -cd * sh, sN = cl * sd - sl * cd * ch, sU = sl * sd + cl * cd * ch;
            if (sU > 0.0) {
                const double za = acos(sU > 1.0 ? 1.0 : sU);
                const double beta = a.domega64[d] * (a.airy ? airy_power(a.freq[f], sE, sN, sU, a.dew, a.dns)
                                                            : exp(a.bcoef64[f] * za * za));
                const double amp = sqrt(beta) * a.amp_scale;
                const double *kp = a.kap64 + ((size_t)f * a.A_all + a.ant[i]) * 3;
                double ph = kp[0] * sE + kp[1] * sN + kp[2] * sU;
                ph -= rint(ph);
                double sn, cs;
                sincospi(2.0 * ph, &sn, &cs);
                out = make_float2((float)(amp * cs), (float)(-amp * sn));
            }
        }
        float *row = E + (size_t)(e / HA_EW) * (2 * HA_EW);
        if (nl < 64 && paired) {
            row[4 * (nl >> 1) + (nl & 1)] = out.x;
            row[4 * (nl >> 1) + 2 + (nl & 1)] = out.y;
        } else if (nl < 64) {
            row[2 * nl] = out.x;
            row[2 * nl + 1] = out.y;
        } else {
            row[128 + 2 * (nl - 64)] = 0.f;
            row[129 + 2 * (nl - 64)] = 0.f;
        }
    }
}

// ------------------------------------------------------------ monopole visibilities
// U[f][t][b] = V_b(x = 1): Eq. rime_discrete for a unit sky, in FP64, for the hour-angle
// geometry.  Per (channel, fringe group) the cell responses P_u(n, d) = dOmega_d A(n, d) K_u(n, d)
// (FP64 phases of the representative pair) are formed once, and pixel r at LST t sits in
// cell n = t k + (R - 1 - r) q, so V_u(t) = sum_d sum_r P_u(t k + (R - 1 - r) q, d) (r
// ascending, d ascending); the sum is written, rounded once to FP32, to every member of the
// group (conjugated for members with the reversed vector).
struct HaMonoArgs {
    int F, D, R, T, B, U, k, q, nh, A_all;
    double lst0, ra_min, dra, dec_min, ddec, lat;
    const double *kap64, *bcoef64, *domega64;
    int airy;
    double dew, dns;
    const double *freq;
    const int *rep;                       // [U][2] antennas of each group's representative pair
    const int *moff, *mem;                // CSR members, b * 2 + reversed
    float *ug;                            // [F][T][U][2] the group's value (nullptr: not kept)
};

__global__ void __launch_bounds__(256) k_ha_monopole(HaMonoArgs a, float *__restrict__ U)
{
    extern __shared__ double smd[];
    double *pr = smd, *pi = pr + a.nh, *ar = pi + a.nh, *ai = ar + a.T;
    const int f = blockIdx.x / a.U, u = blockIdx.x % a.U;
    const double *ki = a.kap64 + ((size_t)f * a.A_all + a.rep[2 * u]) * 3;
    const double *kj = a.kap64 + ((size_t)f * a.A_all + a.rep[2 * u + 1]) * 3;
    const double kd0 = ki[0] - kj[0], kd1 = ki[1] - kj[1], kd2 = ki[2] - kj[2];
    double sl, cl;
    sincos(a.lat, &sl, &cl);
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) ar[t] = ai[t] = 0.0;
    for (int d = 0; d < a.D; ++d) {
        const double dec = a.dec_min + (d + 0.5) * a.ddec;
        double sd, cd;
        sincos(dec, &sd, &cd);
        __syncthreads();
        for (int n = threadIdx.x; n < a.nh; n += blockDim.x) {
            const double H = a.lst0 - (a.ra_min + ((double)((a.R - 1) * a.q - n) + 0.5 * a.q) * (a.dra / a.q));
            double sh, ch;
            sincos(H, &sh, &ch);
            const double sE = -cd * sh, sN = cl * sd - sl * cd * ch, sU = sl * sd + cl * cd * ch;
            double re = 0.0, im = 0.0;
            if (sU > 0.0) {
                const double za = acos(sU > 1.0 ? 1.0 : sU);
                const double w = a.domega64[d] * (a.airy ? airy_power(a.freq[f], sE, sN, sU, a.dew, a.dns)
                                                         : exp(a.bcoef64[f] * za * za));
                double ph = kd0 * sE + kd1 * sN + kd2 * sU;
                ph -= rint(ph);
                double sn, cs;
                sincospi(2.0 * ph, &sn, &cs);
                re = w * cs;
                im = -w * sn;
            }
            pr[n] = re;
            pi[n] = im;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < a.R; ++r) {
                const int n = t * a.k + (a.R - 1 - r) * a.q;
                sr += pr[n];
                si += pi[n];
            }
            ar[t] += sr;
            ai[t] += si;
        }
    }
    __syncthreads();
    const int m0 = a.moff[u], m1 = a.moff[u + 1];
    if (a.ug)
        for (int t = threadIdx.x; t < a.T; t += blockDim.x)
            reinterpret_cast<float2 *>(a.ug)[((size_t)f * a.T + t) * a.U + u] = make_float2((float)ar[t], (float)ai[t]);
    for (int e = threadIdx.x; e < (m1 - m0) * a.T; e += blockDim.x) {
        const int m = m0 + e / a.T, t = e % a.T;
        const int code = a.mem[m], b = code >> 1;
        float2 *dst = reinterpret_cast<float2 *>(U) + ((size_t)f * a.T + t) * a.B + b;
        *dst = make_float2((float)ar[t], (float)((code & 1) ? -ai[t] : ai[t]));
    }
}

// ------------------------------------------------------------ forward operand prep
// ys[f][d][j] = S_f x(r = j + R - nhp, d) for 0 <= r < R, else 0 (j < Ly), split into 16-bit
// hi and lo parts of the operand type.  With m = nhp - 1 - n the sky operand of the forward
// GEMM is B[t][m] = ys[m + t k], increasing in both indices (a Hankel matrix).
template <int ET>
__global__ void k_ha_yprep(HaDev h, const float *__restrict__ x, const unsigned *__restrict__ xmax,
                           uint16_t *__restrict__ ys_hi, uint16_t *__restrict__ ys_lo)
{
    const long long total = (long long)h.F * h.D * (h.Ly / 2);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int jp = 2 * (int)(e % (h.Ly / 2));
        const long long fd = e / (h.Ly / 2);
        const int f = (int)(fd / h.D);
        const float sc = pow2_scale(__uint_as_float(xmax[f]));
        float v[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // element j holds pixel r when j - (nhp - 1 - (R - 1) qc) = r qc (qc cells per pixel)
            const int rr = jp + q - (h.nhp - 1 - (h.R - 1) * h.q);
            const int r = h.q == 1 ? rr : (rr >= 0 && rr % h.q == 0 ? rr / h.q : -1);
            v[q] = (r >= 0 && r < h.R) ? sc * x[fd * h.R + r] : 0.f;
        }
        uint32_t hi, lo;
        Elem<ET>::split(v[0], v[1], hi, lo);
        reinterpret_cast<uint32_t *>(ys_hi)[e] = hi;
        reinterpret_cast<uint32_t *>(ys_lo)[e] = lo;
    }
}

// Hankel image of one (channel, declination) sky strip, per part (hi, lo):
// img[part][j][rho][e] = ys[part][8 j + rho k + e], 16 bytes per (j, rho), j < Jc.
// K known at compile time: thread task (part, j) loads the strip words it needs with
// 16-byte loads and forms the eight chunks in registers (byte permutes for odd shifts).
template <int K, int NT>
__device__ __forceinline__ void build_image(const uint32_t *strip, int Ly, int Jc, uint32_t img_bytes, uint8_t *img,
                                            int t0, int nthr)
{
    constexpr int NW4 = ((7 * K + 7) / 2 + 5) / 4;   // 16-byte words covering elements 8 j .. 8 j + 7 K + 8
    for (int task = t0; task < NT * Jc; task += nthr) {
        const int part = task >= Jc, j = task - part * Jc;
        const uint4 *src = reinterpret_cast<const uint4 *>(strip + part * (Ly / 2)) + j;
        uint32_t w[4 * NW4];
#pragma unroll
        for (int q = 0; q < NW4; ++q) {
            const uint4 v = src[q];
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
        uint4 *dst = reinterpret_cast<uint4 *>(img + (size_t)part * img_bytes + (size_t)j * 128);
#pragma unroll
        for (int rho = 0; rho < 8; ++rho) {
            const int sft = rho * K, ws = sft >> 1;
            uint4 o;
            if (sft & 1) {
                o.x = __byte_perm(w[ws], w[ws + 1], 0x5432);
                o.y = __byte_perm(w[ws + 1], w[ws + 2], 0x5432);
                o.z = __byte_perm(w[ws + 2], w[ws + 3], 0x5432);
                o.w = __byte_perm(w[ws + 3], w[ws + 4], 0x5432);
            } else {
                o = make_uint4(w[ws], w[ws + 1], w[ws + 2], w[ws + 3]);
            }
            dst[rho] = o;
        }
    }
}

// the same for any k: one 16-byte chunk per thread task
template <int NT>
__device__ __forceinline__ void build_image_any(const uint32_t *strip, int Ly, int Jc, int k, uint32_t img_bytes,
                                                uint8_t *img, int t0, int nthr)
{
    const int nch = Jc * 8;
    for (int e = t0; e < NT * nch; e += nthr) {
        const int part = e >= nch, r = e - part * nch, j = r >> 3, rho = r & 7;
        const int s0 = 8 * j + rho * k;
        const uint32_t *w = strip + part * (Ly / 2) + (s0 >> 1);
        uint4 o;
        if (s0 & 1) {
            o.x = __byte_perm(w[0], w[1], 0x5432);
            o.y = __byte_perm(w[1], w[2], 0x5432);
            o.z = __byte_perm(w[2], w[3], 0x5432);
            o.w = __byte_perm(w[3], w[4], 0x5432);
        } else {
            o = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4 *>(img + (size_t)part * img_bytes + (size_t)j * 128 + rho * 16) = o;
    }
}

// ------------------------------------------------------------ forward kernel
// GEMM D[rho][t] = sum_{d, m} A[rho][m] B[t][m] per (M-tile, channel), K = (d, m) with the
// hour-angle cells taken in the order m = nhp - 1 - n.
//   A = P tile, written by the producers into TMEM (the MMA reads it from there): TMEM lane
//       rho = 2 u + (0: Re, 1: Im), two cells per 32-bit column.
//   B = Hankel sky tile B[t][m] = ys[m + t k], never materialised: per (channel, declination)
//       the producers build the image img[j][rho'][e] = ys[8 j + rho' k + e] (rho' < 8,
//       e < 8, 16 bytes per (j, rho')), in which the 8 x 16-byte core matrix of rows
//       t = 8 g .. 8 g + 7 and cells m = 8 jj .. 8 jj + 7 is the 128 contiguous bytes at chunk
//       jj + g k; a K-major descriptor without swizzle (K step 128 B, 8-row step 128 k B)
//       then reads the tile of every chunk straight from the image.
// Work units q in [0, Q), q = (mt F + f) nchunk + d nbc + c (c: 64-cell chunk in m order);
// CTA g takes the contiguous range [Q g / G, Q (g+1) / G).  A segment is the part of one
// (M-tile, channel) pair inside a CTA's range; its partial sum goes to
// vpart[segment][j][t][row] with j the CTA's rank among the segment's contributors.
//   load warp (21): per unit, the E chunk [A][HA_EW] (cells paired) (and, at the first unit of a
//     (channel, declination) group, the two sky strips) by bulk copies;  efull[se] (tx)
//   producers (warps 0-15): four groups of four warps take turns by unit; warp w fills TMEM
//     lanes 32 (w & 3) .. +31 of stage s over all 64 cells (hi, lo), and at the start of a
//     (channel, declination) group its group builds the image;  eempty[se] and full[s]
//     (4 arrivals each: one group)
//   MMA warp (20): 4 K-steps x (1 | 3) MMAs;  commits empty[s], iempty[b] at the end of
//     a group, and accf[q] at the end of a chain of HA_SUB units or a segment
//   epilogue (16-19): adds the chain into the segment's running sum in TMEM columns
//     [2 npad, 3 npad), writes it at the end of a segment;  acce[q] (4 arrivals)
template <int ET, bool X3>
__global__ void __launch_bounds__(HF_THREADS, 1)
k_vis_ha(HaDev h, HaLayout L, const uint16_t *__restrict__ ys_hi, const uint16_t *__restrict__ ys_lo,
         float *__restrict__ vpart, int *__restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    constexpr int NT = X3 ? 2 : 1;
    const uint32_t full0 = base + L.bar_off, empty0 = full0 + 8 * L.nstage;
    const uint32_t efull0 = empty0 + 8 * L.nstage, eempty0 = efull0 + 8 * L.neslot;
    const uint32_t accf0 = eempty0 + 8 * L.neslot, acce0 = accf0 + 16, iempty0 = acce0 + 16;
    const uint32_t misc = L.bar_off + 16 * (L.nstage + L.neslot) + 48;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + misc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < L.nstage; ++s) {
            mbar_init(full0 + 8 * s, HF_PROD_WARPS / HF_PGROUPS);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int s = 0; s < L.neslot; ++s) {
            mbar_init(efull0 + 8 * s, 1);
            mbar_init(eempty0 + 8 * s, HF_PROD_WARPS / HF_PGROUPS);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(accf0 + 8 * q, 1);
            mbar_init(acce0 + 8 * q, 4);
            mbar_init(iempty0 + 8 * q, 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == HF_MMA_WARP) tmem_alloc(su32(tmem_slot), (uint32_t)L.ncols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;
    const int G = gridDim.x;
    const long long q0 = range_lo(h.Q, G, blockIdx.x), q1 = range_lo(h.Q, G, blockIdx.x + 1);
    const uint32_t eb = (uint32_t)h.A * (uint32_t)(HA_EW * 8);    // E chunk bytes
    const uint32_t sb = (uint32_t)h.Lyc * 2u;                     // bytes of one strip part (this chunk)

    if (warp < HF_PROD_WARPS) {
        // ------------------------------------------------------------ producers
        // HF_PGROUPS groups of four warps; group pg builds the units l = q - q0 = pg, pg + HF_PGROUPS, ...,
        // its warp (pg, quarter) the 32 TMEM lanes of that quarter over all 64 cells, as two
        // 16-lane blocks b: lanes 0-7 of a block hold the Re rows and lanes 8-15 the Im rows of
        // groups 16 quarter + 8 b + (0 .. 7) (the drain warps put the rows back in the order
        // 2 u + (Re, Im)).  A thread forms both rows of group 16 quarter + 8 b + lane / 4 on
        // columns 2 (lane % 4) + {0, 1} of every 8 (tcgen05.st.16x256b): one complex product
        // per cell pair for both rows
        const int quarter = warp & 3, pg = warp / 4, gt = 32 * quarter + lane;
        const int ul = 16 * quarter + (lane >> 2);               // block 0's group; block 1's is ul + 8
        const int ccb = 2 * (lane & 3);
        const uint32_t ta_row = tmem_d + ((uint32_t)(32 * quarter) << 16) + (uint32_t)L.abase;
        const int c0 = (int)(q0 % h.nbc);
        const long long per_mt = (long long)h.F * h.nchunk;
        int mt = (int)((q0 + pg) / per_mt);
        long long next_mt = (long long)(mt + 1) * per_mt;
        int c = (int)((q0 + pg) % h.nbc);
        int2 ij0 = h.uij[mt * 64 + ul], ij1 = h.uij[mt * 64 + ul + 8];
        for (long long l = pg; q0 + l < q1; l += HF_PGROUPS) {
            const long long q = q0 + l;
            if (q >= next_mt) {
                mt = (int)(q / per_mt);
                next_mt = (long long)(mt + 1) * per_mt;
                ij0 = h.uij[mt * 64 + ul];
                ij1 = h.uij[mt * 64 + ul + 8];
            }
            const int se = (int)(l % L.neslot), s = (int)(l % L.nstage);
            const uint32_t eph = (uint32_t)((l / L.neslot) & 1), ph = (uint32_t)((l / L.nstage) & 1);
            // a failed wait has raised the abort flag before returning, so after the
            // warp barrier every lane takes the same branch
            mbar_wait_ab(efull0 + 8 * se, eph, abort_flag);
            if (lane == 0 && l >= L.nstage) mbar_wait_ab(empty0 + 8 * s, ph ^ 1u, abort_flag);
            __syncwarp();
            if (*abort_flag) goto done;
            const uint8_t *eslot = gbase + L.e_off + (size_t)se * L.eslot_bytes;
            const bool gstart = (l == 0) || (c == 0);
            if (gstart) {
                // (channel, declination) group index among this CTA's groups; its image buffer
                const long long gi = (c0 + l) / h.nbc;
                const int gb = (int)(gi & 1);
                if (lane == 0 && gi >= 2)
                    mbar_wait_ab(iempty0 + 8 * gb, (uint32_t)(((gi >> 1) - 1) & 1), abort_flag);
                __syncwarp();
                if (*abort_flag) goto done;
                const uint32_t *strip = reinterpret_cast<const uint32_t *>(eslot + eb);
                uint8_t *img = gbase + (size_t)(gb * NT) * L.img_bytes;
                if (h.k == 1) build_image<1, NT>(strip, h.Lyc, h.Jc, L.img_bytes, img, gt, 128);
                else if (h.k == 2) build_image<2, NT>(strip, h.Lyc, h.Jc, L.img_bytes, img, gt, 128);
                else build_image_any<NT>(strip, h.Lyc, h.Jc, h.k, L.img_bytes, img, gt, 128);
            }
            {
                const uint32_t ta = ta_row + (uint32_t)(s * L.acols);
#pragma unroll 1
                for (int b = 0; b < 2; ++b) {
                    const int2 ij = b ? ij1 : ij0;
                    const uint8_t *ei = eslot + (size_t)ij.x * (HA_EW * 8), *ej = eslot + (size_t)ij.y * (HA_EW * 8);
                    const uint32_t tb = ta + ((uint32_t)(16 * b) << 16);
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        // column 8 kq + cc holds cells m = 16 kq + 2 cc (low half) and + 1, i.e.
                        // table cells n + 1 and n with n = 62 - 16 kq - 2 cc: the row's cell pair n / 2
                        uint32_t hw[8], lw[8];
#pragma unroll
                        for (int jr = 0; jr < 2; ++jr) {
                            const int kq = 2 * kh + jr;
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int pc = 31 - 8 * kq - (ccb + e);
                                const float4 a = *reinterpret_cast<const float4 *>(ei + pc * 16);
                                const float4 bq = *reinterpret_cast<const float4 *>(ej + pc * 16);
                                // P = E_i conj(E_j) on the cell pair (n, n + 1), packed: .x cell n
                                // (odd m), .y cell n + 1 (even m)
                                const float2 xa = make_float2(a.x, a.y), ya = make_float2(a.z, a.w);
                                const float2 xb = make_float2(bq.x, bq.y), yb = make_float2(bq.z, bq.w);
                                const float2 re = __ffma2_rn(xa, xb, __fmul2_rn(ya, yb));
                                const float2 mxy = __fmul2_rn(xa, yb);
                                const float2 im = __ffma2_rn(ya, xb, make_float2(-mxy.x, -mxy.y));
                                Elem<ET>::split2(make_float2(re.y, re.x), hw[4 * jr + e], lw[4 * jr + e]);
                                Elem<ET>::split2(make_float2(im.y, im.x), hw[4 * jr + 2 + e], lw[4 * jr + 2 + e]);
                            }
                        }
                        tmem_st_16x256b_x2(tb + 16u * kh, hw);
                        if (X3) tmem_st_16x256b_x2(tb + 32u + 16u * kh, lw);
                    }
                }
                tmem_wait_st();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(eempty0 + 8 * se);
            if (gstart) fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(full0 + 8 * s);
            c = (c + HF_PGROUPS) % h.nbc;
        }
    } else if (warp == HF_LOAD_WARP) {
        // ------------------------------------------------------------ bulk loads of E chunks
        if (lane == 0) {
            int se = 0, last_se = -1;
            uint32_t eph = 0, last_eph = 0;
            bool wrapped = false;
            int f = (int)((q0 / h.nchunk) % h.F), cd = (int)(q0 % h.nchunk);
            for (long long q = q0; q < q1; ++q) {
                if (wrapped && !mbar_wait_ab<64>(eempty0 + 8 * se, eph ^ 1u, abort_flag)) break;
                const int d = cd / h.nbc, c = cd % h.nbc;
                const bool gstart = (q == q0) || (c == 0);
                const float2 *src = h.E + (((size_t)f * h.D + d) * h.nbc + (h.nbc - 1 - c)) * h.A * HA_EW;
                const uint32_t dst = base + L.e_off + (uint32_t)se * L.eslot_bytes;
                // the chunk's LSTs start t0 k elements into the strip (t0 a multiple of 64)
                const size_t row = ((size_t)f * h.D + d) * h.Ly + (size_t)h.t0 * h.k;
                mbar_expect_tx(efull0 + 8 * se, eb + (gstart ? (uint32_t)NT * sb : 0u));
                bulk_g2s(dst, src, eb, efull0 + 8 * se);
                if (gstart) {
                    bulk_g2s(dst + eb, ys_hi + row, sb, efull0 + 8 * se);
                    if (X3) bulk_g2s(dst + eb + sb, ys_lo + row, sb, efull0 + 8 * se);
                }
                last_se = se;
                last_eph = eph;
                if (++se == L.neslot) { se = 0; eph ^= 1u; wrapped = true; }
                if (++cd == h.nchunk) {
                    cd = 0;
                    if (++f == h.F) f = 0;
                }
            }
            // copies still in flight must land before the CTA exits (bounded); without an
            // abort the producers have already waited for every one of them
            if (*abort_flag && last_se >= 0) {
                for (int k = 0; k < L.neslot; ++k) {
                    int s2 = last_se - k;
                    uint32_t p2 = last_eph;
                    if (s2 < 0) { s2 += L.neslot; p2 ^= 1u; }
                    if ((long long)k < q1 - q0) mbar_drain(efull0 + 8 * s2, p2);
                }
            }
        }
    } else if (warp == HF_MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, h.npad, Elem<ET>::kFmt);
            const uint32_t sbo = 128u * (uint32_t)h.k;
            int s = 0, last_s = -1, gb = 0;
            uint32_t ph = 0, last_ph = 0;
            long long nacc = 0, ngrp = 0;
            int local = 0, cd = (int)(q0 % h.nchunk);
            for (long long q = q0; q < q1; ++q, cd = (cd + 1 == h.nchunk) ? 0 : cd + 1) {
                const int c = cd % h.nbc;
                if (q == q0 || cd == 0) local = 0;
                if (q == q0 || c == 0) gb = (int)(ngrp++ & 1);
                const bool chain_first = (local % HA_SUB) == 0;
                const int qa = (int)(nacc & 1);
                if (chain_first && nacc >= 2 &&
                    !mbar_wait_ab<64>(acce0 + 8 * qa, (uint32_t)(((nacc >> 1) - 1) & 1), abort_flag))
                    goto mma_done;
                if (!mbar_wait_ab<32>(full0 + 8 * s, ph, abort_flag)) goto mma_done;
                tc_fence_after();
                {
                    const uint32_t dacc = tmem_d + (uint32_t)(qa * h.npad);
                    const uint32_t ta = tmem_d + (uint32_t)(L.abase + s * L.acols);
                    const uint32_t ib = base + (uint32_t)(gb * NT) * L.img_bytes + (uint32_t)(8 * c) * 128u;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t dbh = sdesc_none(ib + 256u * kk, 128u, sbo);
                        mma_ts(dacc, ta + 8u * kk, dbh, idesc, (chain_first && kk == 0) ? 0u : 1u);
                        if (X3) {
                            mma_ts(dacc, ta + 8u * kk, sdesc_none(ib + L.img_bytes + 256u * kk, 128u, sbo), idesc, 1u);
                            mma_ts(dacc, ta + 32u + 8u * kk, dbh, idesc, 1u);
                        }
                    }
                }
                mma_commit(empty0 + 8 * s);
                if (q == q1 - 1 || c == h.nbc - 1) mma_commit(iempty0 + 8 * gb);
                last_s = s;
                last_ph = ph;
                if (++s == L.nstage) { s = 0; ph ^= 1u; }
                ++local;
                const bool seg_last = (q == q1 - 1) || (cd == h.nchunk - 1);
                if ((local % HA_SUB) == 0 || seg_last) {
                    mma_commit(accf0 + 8 * qa);
                    ++nacc;
                }
            }
        mma_done:
            if (*abort_flag && last_s >= 0) mbar_drain(empty0 + 8 * last_s, last_ph);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps HF_EPI_WARP0 ..)
        // TMEM lane 32 quarter + 16 b + 8 part + j holds row 2 u + part of group
        // u = 16 quarter + 8 b + j (the producers' 16-lane blocks)
        const int quarter = warp & 3, lb = lane & 15;
        const int row = 32 * quarter + 16 * (lane >> 4) + 2 * (lb & 7) + (lb >> 3);
        // the running sum of the segment lives in TMEM columns [2 npad, 3 npad)
        const uint32_t tsum = tmem_d + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(2 * h.npad);
        {
            float z[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = 0.f;
            for (int c16 = 0; c16 < h.npad; c16 += 16) tmem_st16(tsum + (uint32_t)c16, z);
        }
        long long nacc = 0;
        int local = 0, seg = (int)(q0 / h.nchunk), c = (int)(q0 % h.nchunk);
        for (long long q = q0; q < q1; ++q) {
            if (q != q0 && ++c == h.nchunk) { c = 0; ++seg; }
            if (q == q0 || c == 0) local = 0;
            ++local;
            const bool seg_last = (q == q1 - 1) || (c == h.nchunk - 1);
            if (!((local % HA_SUB) == 0 || seg_last)) continue;
            const int qa = (int)(nacc & 1);
            mbar_wait_ab<128>(accf0 + 8 * qa, (uint32_t)((nacc >> 1) & 1), abort_flag);
            __syncwarp();
            if (*abort_flag) goto done;
            tc_fence_after();
            const uint32_t taddr = tmem_d + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(qa * h.npad);
            float *dst = nullptr;
            if (seg_last) {
                const int jrank = blockIdx.x - cta_of((long long)seg * h.nchunk, h.Q, G);
                dst = vpart + ((size_t)seg * h.J + jrank) * h.npad * 128 + row;
            }
            for (int c16 = 0; c16 < h.npad; c16 += 16) {
                float v[16], a[16];
                tmem_ld16(taddr + (uint32_t)c16, v);
                tmem_ld16(tsum + (uint32_t)c16, a);
#pragma unroll
                for (int j = 0; j < 16; ++j) a[j] += v[j];
                if (seg_last) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (c16 + j < h.T) dst[(size_t)(c16 + j) * 128] = a[j];
                        a[j] = 0.f;
                    }
                }
                tmem_st16(tsum + (uint32_t)c16, a);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * qa);
            ++nacc;
        }
    }
done:
    __syncthreads();
    if (*abort_flag && tid == 0) atomicExch(status, (int)FM_ERR_TIMEOUT);
    if (warp == HF_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem_d, (uint32_t)L.ncols);
    }
}

// Sum of the forward partials in fixed order, unscaled, expanded to every baseline.
// CTA (segment, LST block of HA_VF_T): the contributors' partials of the segment's 128
// rows are added into shared memory, then every baseline of the segment's groups gets
// its (possibly conjugated) value, written coalesced over baselines.  With dc != nullptr
// the monopole term c_f U[f][t][b] (c_f = dc[f * dcs]) is added in the same write.
constexpr int HA_VF_T = 8;

__global__ void __launch_bounds__(256) k_ha_vfinish(HaDev h, int B, const float *__restrict__ vpart,
                                                    const int *__restrict__ ncontrib, const int *__restrict__ bmap,
                                                    const unsigned *__restrict__ xmax, float sp,
                                                    const float *__restrict__ dc, long long dcs,
                                                    const float *__restrict__ U, float *__restrict__ vis)
{
    __shared__ float sv[128][HA_VF_T];
    const int seg = blockIdx.x, mt = seg / h.F, f = seg % h.F;
    const int t0 = blockIdx.y * HA_VF_T, tn = min(HA_VF_T, h.T - t0);
    const int nc = ncontrib[seg];
    for (int e = threadIdx.x; e < 128 * HA_VF_T; e += blockDim.x) {
        const int row = e % 128, tl = e / 128;
        float a = 0.f;
        if (tl < tn) {      // the contributors' rows in rank order, four loads ahead
            const float *src = vpart + ((size_t)seg * h.J * h.npad + t0 + tl) * 128 + row;
            const size_t js = (size_t)h.npad * 128;
            for (int j0 = 0; j0 < nc; j0 += 4) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = j0 + u < nc ? src[(size_t)(j0 + u) * js] : 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j0 + u < nc) a += v[u];
            }
        }
        sv[row][tl] = a;
    }
    __syncthreads();
    const float sc = 1.f / (sp * pow2_scale(__uint_as_float(xmax[f])));
    const float cf = dc ? dc[(size_t)f * dcs] : 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const int code = bmap[b], u = code >> 1;
        if ((u >> 6) != mt) continue;
        const int row = 2 * (u & 63);
        const float sgn = (code & 1) ? -1.f : 1.f;
        for (int tl = 0; tl < tn; ++tl) {
            const size_t e = ((size_t)f * h.Tt + h.t0 + t0 + tl) * B + b;
            // explicit roundings: the chi^2 epilogue forms the same values (HaVSrc)
            float2 v = make_float2(__fmul_rn(sv[row][tl], sc), __fmul_rn(sgn * sv[row + 1][tl], sc));
            if (dc) {
                const float2 u2 = reinterpret_cast<const float2 *>(U)[e];
                v.x = __fmaf_rn(cf, u2.x, v.x);
                v.y = __fmaf_rn(cf, u2.y, v.y);
            }
            reinterpret_cast<float2 *>(vis)[e] = v;
        }
    }
}

// largest |x| of each channel as float bits (non-negative floats order like their bit
// patterns): blockIdx.y = channel, the CTAs of a channel split its pixels
__global__ void __launch_bounds__(256) k_ha_xmax(int npix, const float *__restrict__ x, unsigned *__restrict__ xmax)
{
    __shared__ float red[256];
    const int f = blockIdx.y;
    float m = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[(size_t)f * npix + p]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(xmax + f, __float_as_uint(red[0]));
}

// ------------------------------------------------------------ adjoint operand prep
// Q_u(f, t) = sum of omega over the group's members (conjugated for reversed ones) and
// the largest |Re|, |Im| per (channel, LST).
__global__ void __launch_bounds__(256) k_ha_qsum(HaDev h, int B, const float *__restrict__ omega,
                                                 const int *__restrict__ moff, const int *__restrict__ mem,
                                                 float *__restrict__ q32, float *__restrict__ qmax_ft)
{
    // one CTA per (channel, LST): the omega row is staged in shared memory, each thread
    // sums the members of its groups, and the CTA records its maximum
    extern __shared__ float som[];                  // [2 B]
    __shared__ float red[256];
    const int ft = blockIdx.x, f = ft / h.Tt;
    const float *om = omega + (size_t)ft * B * 2;
    for (int e = threadIdx.x; e < 2 * B; e += blockDim.x) som[e] = om[e];
    __syncthreads();
    float mx = 0.f;
    for (int u = threadIdx.x; u < h.U; u += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int m = moff[u]; m < moff[u + 1]; ++m) {
            const int code = mem[m], b = code >> 1;
            re += som[2 * b];
            im += (code & 1) ? -som[2 * b + 1] : som[2 * b + 1];
        }
        q32[((size_t)ft * h.U + u) * 2] = re;
        q32[((size_t)ft * h.U + u) * 2 + 1] = im;
        mx = fmaxf(mx, fmaxf(fabsf(re), fabsf(im)));
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) qmax_ft[ft] = red[0];
    (void)f;
}

// One CTA per (channel, K chunk): the swizzled B tile [npad rows t][64 rho] of the
// adjoint for the LSTs t0 + t, t < T, of the current chunk, hi then (x3) lo, ready for one
// bulk copy; the power-of-two scale is the chunk's.
template <int ET, bool X3>
__global__ void k_ha_qimg(HaDev h, const float *__restrict__ q32, const float *__restrict__ qmax_ft,
                          float *__restrict__ qscale, uint8_t *__restrict__ qimg)
{
    constexpr int NT = X3 ? 2 : 1;
    const int f = blockIdx.x / h.nkq, kq = blockIdx.x % h.nkq;
    __shared__ float smx;
    if (threadIdx.x < 32) {
        float m = 0.f;
        for (int t = threadIdx.x; t < h.T; t += 32) m = fmaxf(m, qmax_ft[(size_t)f * h.Tt + h.t0 + t]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) smx = m;
    }
    __syncthreads();
    const float sc = pow2_scale(smx);
    if (kq == 0 && threadIdx.x == 0) qscale[f] = sc;
    const uint32_t b_bytes = (uint32_t)h.npad * 128u;
    uint8_t *img = qimg + ((size_t)f * h.nkq + kq) * NT * b_bytes;
    for (int e = threadIdx.x; e < h.npad * 8; e += blockDim.x) {
        const int t = e >> 3, ch = e & 7;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = 32 * kq + 4 * ch + q;
            float re = 0.f, im = 0.f;
            if (t < h.T && u < h.U) {
                const float *p = q32 + (((size_t)f * h.Tt + h.t0 + t) * h.U + u) * 2;
                re = p[0] * sc;
                im = p[1] * sc;
            }
            Elem<ET>::split(re, im, hw[q], lw[q]);
        }
        const uint32_t off = sw128_off(t, ch);
        *reinterpret_cast<uint4 *>(img + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if (X3) *reinterpret_cast<uint4 *>(img + b_bytes + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// ------------------------------------------------------------ adjoint kernel
// Items (f, d), CTA g takes items g, g + G, ...; per item the nhp / 128 M-tiles of 128
// hour-angle cells, per M-tile the nkq K chunks of 64 rho = 32 groups.
//   table warp (21): per M-tile, the two E chunks (bulk, efull[se])
//   Q warp (22): per K chunk, the Q tile into the stage's B part (bulk, bfull[s])
//   producers (0-15): thread (row n = tid & 127, quarter = tid >> 7) writes the 8 groups
//     8 quarter .. +7 of row n into TMEM lane n (A operand of stage s: 8 columns hi, 8 lo);
//     then full[s]
//   MMA warp (20): D[n][t] of the M-tile into TMEM set (M-tile count & 1);  accf[q]
//   epilogue (16-19 and 23-26, one set per 32-LST half): the diagonal sums over the
//     M-tiles of the item (see below), one output row xbar(., d) per item.
template <int ET, bool X3>
__global__ void __launch_bounds__(HA_ADJ_THREADS, 1)
k_adj_ha(HaDev h, HaLayout L, const uint8_t *__restrict__ qimg, const float *__restrict__ qscale, float sp,
         float *__restrict__ xbar, int *__restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    constexpr int NT = X3 ? 2 : 1;
    const uint32_t full0 = base + L.bar_off, empty0 = full0 + 8 * L.nstage;
    const uint32_t efull0 = empty0 + 8 * L.nstage, eempty0 = efull0 + 8 * L.neslot;
    const uint32_t accf0 = eempty0 + 8 * L.neslot, acce0 = accf0 + 16;
    const uint32_t bfull0 = acce0 + 16;
    const uint32_t misc = L.bar_off + 16 * (L.nstage + L.neslot) + 32 + 8 * L.nstage;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + misc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the groups' table rows as byte offsets within an E chunk
    int2 *suij = reinterpret_cast<int2 *>(gbase + L.v_off + ((size_t)2 * 32 * (128 + 64 * h.k + 1) + 4 * 128) * 4);
    for (int e = tid; e < 32 * h.nkq; e += blockDim.x) {
        const int2 ij = h.uij[e];
        suij[e] = make_int2(ij.x * (HA_EW * 8), ij.y * (HA_EW * 8));
    }
    if (tid == 0) {
        for (int s = 0; s < L.nstage; ++s) {
            mbar_init(full0 + 8 * s, HA_PROD_WARPS);
            mbar_init(empty0 + 8 * s, 1);
            mbar_init(bfull0 + 8 * s, 1);
        }
        for (int s = 0; s < L.neslot; ++s) {
            mbar_init(efull0 + 8 * s, 1);
            mbar_init(eempty0 + 8 * s, HA_PROD_WARPS);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(accf0 + 8 * q, 1);
            mbar_init(acce0 + 8 * q, 8);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == HA_MMA_WARP) tmem_alloc(su32(tmem_slot), (uint32_t)L.ncols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;
    const int nitem = h.F * h.D, nmta = h.nhp / 128;
    const uint32_t echunk = (uint32_t)h.A * (uint32_t)(HA_EW * 8);

    if (warp < HA_PROD_WARPS) {
        // ------------------------------------------------------------ producers
        const int n = tid & 127, qq = tid >> 7;
        int s = 0, se = 0;
        uint32_t ph = 0, eph = 0;
        bool wrapped = false;
        for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
            for (int mt = 0; mt < nmta; ++mt) {
                mbar_wait_ab(efull0 + 8 * se, eph, abort_flag);
                __syncwarp();
                if (*abort_flag) goto done;
                // shared address of this row's cell in the slot's first table row
                const uint32_t es = base + L.e_off + (uint32_t)se * L.eslot_bytes + (uint32_t)(n >> 6) * echunk +
                                    (uint32_t)(n & 63) * 8u;
                for (int kq = 0; kq < h.nkq; ++kq) {
                    if (lane == 0 && wrapped) mbar_wait_ab(empty0 + 8 * s, ph ^ 1u, abort_flag);
                    __syncwarp();
                    if (*abort_flag) goto done;
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int2 ij = suij[32 * kq + 8 * qq + q];
                        const float2 a = lds_f2(es + (uint32_t)ij.x), b = lds_f2(es + (uint32_t)ij.y);
                        Elem<ET>::split2(make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y)), hw[q], lw[q]);
                    }
                    // TMEM lane n (= 32 (warp & 3) + lane), columns 8 qq .. 8 qq + 7 of stage s
                    const uint32_t ta = tmem_d + ((uint32_t)(32 * (warp & 3)) << 16) +
                                        (uint32_t)(L.abase + s * L.acols + 8 * qq);
                    tmem_st8(ta, hw);
                    if (X3) tmem_st8(ta + 32u, lw);
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full0 + 8 * s);
                    if (++s == L.nstage) { s = 0; ph ^= 1u; wrapped = true; }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(eempty0 + 8 * se);
                if (++se == L.neslot) { se = 0; eph ^= 1u; }
            }
        }
    } else if (warp == HA_LOAD_WARP) {
        // ------------------------------------------------------------ bulk loads of E
        if (lane == 0) {
            int se = 0, last_se = -1;
            uint32_t eph = 0, last_eph = 0;
            bool ewrapped = false;
            long long nse = 0;
            for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
                const int f = it / h.D, d = it % h.D;
                for (int mt = 0; mt < nmta; ++mt) {
                    if (ewrapped && !mbar_wait_ab<64>(eempty0 + 8 * se, eph ^ 1u, abort_flag)) goto eload_done;
                    const float2 *src = h.Ea + (((size_t)f * h.D + d) * h.nbc + 2 * mt) * h.A * HA_EW;
                    const uint32_t dst = base + L.e_off + (uint32_t)se * L.eslot_bytes;
                    mbar_expect_tx(efull0 + 8 * se, 2 * echunk);
                    bulk_g2s(dst, src, echunk, efull0 + 8 * se);
                    bulk_g2s(dst + echunk, src + (size_t)h.A * HA_EW, echunk, efull0 + 8 * se);
                    last_se = se;
                    last_eph = eph;
                    ++nse;
                    if (++se == L.neslot) { se = 0; eph ^= 1u; ewrapped = true; }
                }
            }
        eload_done:
            // copies in flight land before the CTA exits (bounded)
            if (*abort_flag) {
                for (int k = 0; k < L.neslot && k < nse; ++k) {
                    int s2 = last_se - k;
                    uint32_t p2 = last_eph;
                    if (s2 < 0) { s2 += L.neslot; p2 ^= 1u; }
                    mbar_drain(efull0 + 8 * s2, p2);
                }
            }
        }
    } else if (warp == HA_QLOAD_WARP) {
        // ------------------------------------------------------------ bulk loads of Q tiles
        if (lane == 0) {
            int s = 0, last_s = -1;
            uint32_t ph = 0, last_ph = 0;
            bool wrapped = false;
            long long ns = 0;
            const uint32_t bbytes = NT * L.b_bytes;
            for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
                const int f = it / h.D;
                for (int mt = 0; mt < nmta; ++mt)
                    for (int kq = 0; kq < h.nkq; ++kq) {
                        if (wrapped && !mbar_wait_ab<64>(empty0 + 8 * s, ph ^ 1u, abort_flag)) goto qload_done;
                        mbar_expect_tx(bfull0 + 8 * s, bbytes);
                        bulk_g2s(base + (uint32_t)s * L.stage_bytes,
                                 qimg + ((size_t)f * h.nkq + kq) * bbytes, bbytes, bfull0 + 8 * s);
                        last_s = s;
                        last_ph = ph;
                        ++ns;
                        if (++s == L.nstage) { s = 0; ph ^= 1u; wrapped = true; }
                    }
            }
        qload_done:
            if (*abort_flag) {
                for (int k = 0; k < L.nstage && k < ns; ++k) {
                    int s2 = last_s - k;
                    uint32_t p2 = last_ph;
                    if (s2 < 0) { s2 += L.nstage; p2 ^= 1u; }
                    mbar_drain(bfull0 + 8 * s2, p2);
                }
            }
        }
    } else if (warp == HA_MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, h.npad, Elem<ET>::kFmt);
            int s = 0, last_s = -1;
            uint32_t ph = 0, last_ph = 0;
            long long nacc = 0;
            for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
                for (int mt = 0; mt < nmta; ++mt) {
                    const int qa = (int)(nacc & 1);
                    if (nacc >= 2 && !mbar_wait_ab<64>(acce0 + 8 * qa, (uint32_t)(((nacc >> 1) - 1) & 1), abort_flag))
                        goto mma_done;
                    const uint32_t dacc = tmem_d + (uint32_t)(qa * h.npad);
                    for (int kq = 0; kq < h.nkq; ++kq) {
                        if (!mbar_wait_ab<32>(full0 + 8 * s, ph, abort_flag)) goto mma_done;
                        if (!mbar_wait_ab<32>(bfull0 + 8 * s, ph, abort_flag)) goto mma_done;
                        tc_fence_after();
                        const uint32_t b_hi = base + (uint32_t)s * L.stage_bytes, b_lo = b_hi + L.b_bytes;
                        const uint32_t ta = tmem_d + (uint32_t)(L.abase + s * L.acols);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t dbh = sdesc_sw128(b_hi + 32u * kk);
                            mma_ts(dacc, ta + 8u * kk, dbh, idesc, (kq == 0 && kk == 0) ? 0u : 1u);
                            if (X3) {
                                mma_ts(dacc, ta + 8u * kk, sdesc_sw128(b_lo + 32u * kk), idesc, 1u);
                                mma_ts(dacc, ta + 32u + 8u * kk, dbh, idesc, 1u);
                            }
                        }
                        mma_commit(empty0 + 8 * s);
                        last_s = s;
                        last_ph = ph;
                        if (++s == L.nstage) { s = 0; ph ^= 1u; }
                    }
                    mma_commit(accf0 + 8 * qa);
                    ++nacc;
                }
            }
        mma_done:
            if (*abort_flag && last_s >= 0) mbar_drain(empty0 + 8 * last_s, last_ph);
        }
    } else if ((warp >= HA_EPI_WARP0 && warp < HA_EPI_WARP0 + 4) || warp >= HA_EPI2_WARP0) {
        // ------------------------------------------------------------ epilogue (warps 16-19, 23-26)
        // Two sets of four warps, set eh for the LSTs [32 eh, 32 eh + 32).  Per M-tile a set
        // moves its half of the accumulator D[n][t] into its shared tile sk[t][pk + n] (row
        // stride skw = 128 + 2 pk + 1, pk = 32 k zero cells on both sides of each row); thread
        // et then adds, for its outputs r = et + 128 j, the entries on the diagonal
        // n = t k + R - 1 - r - 128 mt: 32 unconditional loads (the diagonal leaves [0, 128)
        // only into the zero margins) into four partial sums, added in a fixed order.  At the
        // end of an item set 1 hands its sums to set 0 through shared memory, which adds them
        // and stores x-bar.  Named barrier 1 + eh spans a set, barrier 3 both sets; the
        // OR-reduced form of barrier 3 decides a wind-down for all eight warps at once.
        const int eh = warp >= HA_EPI2_WARP0;
        const int quarter = warp & 3, et = 32 * quarter + lane;          // TMEM lane = n = et
        const int pk = 32 * h.k, skw = 128 + 2 * pk + 1;
        float *sk = reinterpret_cast<float *>(gbase + L.v_off) + (size_t)eh * 32 * skw;   // [32][skw]
        float *xs1 = reinterpret_cast<float *>(gbase + L.v_off) + (size_t)2 * 32 * skw;  // [4][128]
        for (int e = et; e < 32 * skw; e += 128) sk[e] = 0.f;
        bar_or(1 + eh, 128, false);
        const int t0 = 32 * eh;
        long long nacc = 0;
        for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
            const int f = it / h.D, d = it % h.D;
            float xr[4] = {0.f, 0.f, 0.f, 0.f};      // outputs r = et + 128 j (R <= 512)
            bool stop = false;
            for (int mt = 0; mt < nmta; ++mt, ++nacc) {
                const int qa = (int)(nacc & 1);
                mbar_wait_ab<128>(accf0 + 8 * qa, (uint32_t)((nacc >> 1) & 1), abort_flag);
                __syncwarp();
                if (bar_or(3, 256, *abort_flag != 0)) { stop = true; break; }
                tc_fence_after();
                const uint32_t taddr = tmem_d + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(qa * h.npad);
                const int c0 = (h.R - 1) * h.q - 128 * mt + h.t0 * h.k;      // n = t k + c0 - r q (t in the chunk)
                if (t0 < h.T) {
                    // LST columns t >= T hold zeros (zero residual rows); those past npad are
                    // not loaded and set to zero here
                    float v[32];
                    tmem_ld16(taddr + (uint32_t)t0, v);
                    if (t0 + 16 < h.npad) {
                        tmem_ld16(taddr + (uint32_t)(t0 + 16), v + 16);
                    } else {
#pragma unroll
                        for (int q = 16; q < 32; ++q) v[q] = 0.f;
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce0 + 8 * qa);   // the accumulator is read
#pragma unroll
                    for (int q = 0; q < 32; ++q) sk[q * skw + pk + et] = v[q];
                    bar_or(1 + eh, 128, false);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (et + 128 * j >= h.R) break;
                        // entry (q, nb0 + q k), q < 32; nothing of [0, 128) on the diagonal when
                        // nb0 + 31 k < 0 or nb0 >= 128, otherwise every entry lies in the row
                        // or its margins
                        const int nb0 = t0 * h.k + c0 - (et + 128 * j) * h.q;
                        if (nb0 + 31 * h.k < 0 || nb0 >= 128) continue;
                        const float *col = sk + pk + nb0;
                        const int st = skw + h.k;
                        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            a0 += col[q * st];
                            a1 += col[(q + 1) * st];
                            a2 += col[(q + 2) * st];
                            a3 += col[(q + 3) * st];
                        }
                        xr[j] += (a0 + a1) + (a2 + a3);
                    }
                    bar_or(1 + eh, 128, false);
                } else {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce0 + 8 * qa);
                }
            }
            if (stop) break;
            if (eh) {
#pragma unroll
                for (int j = 0; j < 4; ++j) xs1[j * 128 + et] = xr[j];
            }
            bar_or(3, 256, false);
            if (!eh) {
                const float sc = 1.f / (sp * qscale[f]);
                float *xo = xbar + ((size_t)f * h.D + d) * h.R;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (et + 128 * j < h.R) {
                        // later LST chunks add to the earlier ones' sum (stream order)
                        const float v = (xr[j] + xs1[j * 128 + et]) * sc;
                        xo[et + 128 * j] = h.t0 > 0 ? xo[et + 128 * j] + v : v;
                    }
            }
            bar_or(3, 256, false);
        }
    }
done:
    __syncthreads();
    if (*abort_flag && tid == 0) atomicExch(status, (int)FM_ERR_TIMEOUT);
    if (warp == HA_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem_d, (uint32_t)L.ncols);
    }
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

HaDev make_dev(const Ctx &c)
{
    const HaState &s = c.ha;
    HaDev h;
    h.F = c.F; h.D = c.D; h.T = c.T; h.R = c.R; h.A = s.nant + 1; h.U = s.U; h.k = s.k; h.q = s.q;
    h.nhp = s.nhp; h.nbc = s.nbc; h.npad = s.npad; h.Ly = s.Ly; h.Jc = s.Jc;
    h.Tt = c.T; h.t0 = 0; h.Lyc = s.Lyc; h.T = c.T < HA_TCHUNK ? c.T : HA_TCHUNK;
    h.nchunk = c.D * s.nbc; h.nmt = s.nmt; h.nkq = s.nkq; h.J = s.J;
    h.Q = (long long)s.nmt * c.F * h.nchunk;
    h.E = s.E; h.Ea = s.Ea; h.uij = s.uij;
    return h;
}

bool x3_of(int prec) { return prec == FM_PREC_BF16X3 || prec == FM_PREC_FP16X3; }
bool f16_of(int prec) { return prec == FM_PREC_FP16X1 || prec == FM_PREC_FP16X3; }

// adjoint scratch: the two epilogue sets' tiles sk [32][128 + 64 k + 1] (32 k zero cells on
// each side of a row), set 1's partial sums [4][128] and the group pairs [32 nkq]
uint32_t adj_scratch_bytes(const Ctx &c)
{
    return (2u * 32u * (128u + 64u * (uint32_t)c.ha.k + 1u) + 4u * 128u) * 4u + 32u * (uint32_t)c.ha.nkq * 8u;
}

// TMEM columns of both kernels: the accumulators (two sets, and the forward's running sum),
// then `nstage` A stages of 32 columns per part
void tmem_layout(const Ctx &c, bool x3, int nacc_sets, int nstage, HaLayout &L)
{
    L.nstage = nstage;
    L.acols = (x3 ? 2 : 1) * 32;
    L.abase = (nacc_sets * c.ha.npad + 31) / 32 * 32;
    L.ncols = 512;
}

// forward: two image buffers (hi, lo), then as many table slots (E chunk [A][HA_EW] and
// the two sky strips) as fit, up to 8, at least 2
bool make_layout_fwd(const Ctx &c, bool x3, HaLayout &L)
{
    const int nt = x3 ? 2 : 1;
    tmem_layout(c, x3, 3, HA_NSTAGE_FWD, L);
    if (L.abase + L.nstage * L.acols > L.ncols) return false;
    L.b_bytes = 0;
    L.stage_bytes = 0;
    L.img_bytes = (uint32_t)c.ha.Jc * 128u;
    L.eslot_bytes = (uint32_t)(c.ha.nant + 1) * (uint32_t)(HA_EW * 8) + (uint32_t)nt * (uint32_t)c.ha.Lyc * 2u;
    L.e_off = 2u * (uint32_t)nt * L.img_bytes;
    const size_t bars = 16 * (size_t)L.nstage + 48 + 16;
    L.neslot = 8;
    while (L.neslot >= 2 && (size_t)L.e_off + (size_t)L.neslot * L.eslot_bytes + bars + 16 * L.neslot >
                                (size_t)HA_SMEM_BUDGET)
        --L.neslot;
    if (L.neslot < 2) return false;
    L.v_off = L.e_off + (uint32_t)L.neslot * L.eslot_bytes;
    L.bar_off = L.v_off;
    L.smem = 1024 + (size_t)L.bar_off + 16 * (L.nstage + L.neslot) + 48 + 16;
    return L.smem <= 227 * 1024;
}

// adjoint: HA_NSTAGE residual tiles (B operand), table slots of two E chunks (up to 4, at
// least 2) and the epilogue's scratch
bool make_layout_adj(const Ctx &c, bool x3, HaLayout &L)
{
    const int nt = x3 ? 2 : 1;
    tmem_layout(c, x3, 2, HA_NSTAGE, L);
    if (L.abase + L.nstage * L.acols > L.ncols) return false;
    L.b_bytes = (uint32_t)c.ha.npad * 128u;
    L.stage_bytes = (uint32_t)nt * L.b_bytes;
    L.img_bytes = 0;
    L.eslot_bytes = 2u * (uint32_t)(c.ha.nant + 1) * (uint32_t)(HA_EW * 8);
    const uint32_t vbytes = (adj_scratch_bytes(c) + 15) / 16 * 16;
    const size_t bars = 24 * (size_t)L.nstage + 32 + 16;
    L.e_off = (uint32_t)L.nstage * L.stage_bytes;
    L.neslot = 4;
    while (L.neslot >= 2 &&
           (size_t)L.e_off + (size_t)L.neslot * L.eslot_bytes + vbytes + bars + 16 * L.neslot > (size_t)HA_SMEM_BUDGET)
        --L.neslot;
    if (L.neslot < 2) return false;
    L.v_off = L.e_off + (uint32_t)L.neslot * L.eslot_bytes;
    L.bar_off = L.v_off + vbytes;
    L.smem = 1024 + (size_t)L.bar_off + 24 * L.nstage + 16 * L.neslot + 32 + 16;
    return L.smem <= 227 * 1024;
}

template <int ET, bool X3>
fm_status vis_ha_launch(Ctx &c, const HaDev &h, const float *x, float *vis, cudaStream_t st, const float *dc,
                        long long dcs, bool xmax_ready, bool strips_ready, bool partials_only)
{
    HaState &s = c.ha;
    HaLayout L;
    if (!make_layout_fwd(c, X3, L)) {
        set_error("hour-angle forward tiles exceed shared memory");
        return FM_ERR_UNSUPPORTED;
    }
    uint16_t *ys_hi = s.ys, *ys_lo = s.ys + (size_t)c.F * c.D * s.Ly;
    if (!xmax_ready) {
        FM_CK(cudaMemsetAsync(s.xmax, 0, sizeof(unsigned) * c.F, st));
        k_ha_xmax<<<dim3(cdiv(c.npix, 256 * 8), c.F), 256, 0, st>>>(c.npix, x, s.xmax);
        FM_CK_LAUNCH();
    }
    if (!strips_ready) {
        k_ha_yprep<ET><<<1024, 256, 0, st>>>(h, x, s.xmax, ys_hi, ys_lo);
        FM_CK_LAUNCH();
    }
    FM_CK(smem_opt_in(k_vis_ha<ET, X3>));
    // one pass per chunk of at most HA_TCHUNK LSTs (the partial sums are reused)
    for (int t0 = 0; t0 < c.T; t0 += HA_TCHUNK) {
        HaDev hc = h;
        hc.t0 = t0;
        hc.T = c.T - t0 < HA_TCHUNK ? c.T - t0 : HA_TCHUNK;
        FM_TRY(profiled(c, 0, st, [&]() -> fm_status {
            k_vis_ha<ET, X3><<<s.grid, HF_THREADS, L.smem, st>>>(hc, L, ys_hi, ys_lo, s.vpart, c.status);
            FM_CK_LAUNCH();
            return FM_OK;
        }));
        if (partials_only) {
            if (c.T > HA_TCHUNK) {
                set_error("the forward's partial sums hold one pass of at most %d LSTs", HA_TCHUNK);
                return FM_ERR_STATE;
            }
            continue;
        }
        k_ha_vfinish<<<dim3(s.nmt * c.F, cdiv(hc.T, HA_VF_T)), 256, 0, st>>>(hc, c.B, s.vpart, s.ncontrib, s.bmap,
                                                                             s.xmax, s.sp, dc, dcs, c.dc_u, vis);
        FM_CK_LAUNCH();
    }
    return FM_OK;
}

template <int ET, bool X3>
fm_status adj_ha_launch(Ctx &c, const HaDev &h, const float *omega, float *xbar, cudaStream_t st, bool q_ready)
{
    HaState &s = c.ha;
    HaLayout L;
    if (!make_layout_adj(c, X3, L)) {
        set_error("hour-angle adjoint tiles exceed shared memory");
        return FM_ERR_UNSUPPORTED;
    }
    if (!q_ready) {
        k_ha_qsum<<<c.F * c.T, 256, sizeof(float) * 2 * (size_t)c.B, st>>>(h, c.B, omega, s.moff, s.mem, s.q32,
                                                                            s.qmax_ft);
        FM_CK_LAUNCH();
    }
    int grid = s.grid_adj > 0 ? s.grid_adj : sm_count();
    if (grid > c.F * c.D) grid = c.F * c.D;
    FM_CK(smem_opt_in(k_adj_ha<ET, X3>));
    // one pass per chunk of at most HA_TCHUNK LSTs; passes after the first add to xbar
    for (int t0 = 0; t0 < c.T; t0 += HA_TCHUNK) {
        HaDev hc = h;
        hc.t0 = t0;
        hc.T = c.T - t0 < HA_TCHUNK ? c.T - t0 : HA_TCHUNK;
        k_ha_qimg<ET, X3><<<c.F * s.nkq, 256, 0, st>>>(hc, s.q32, s.qmax_ft, s.qscale, s.qimg);
        FM_CK_LAUNCH();
        FM_TRY(profiled(c, 1, st, [&]() -> fm_status {
            k_adj_ha<ET, X3><<<grid, HA_ADJ_THREADS, L.smem, st>>>(hc, L, s.qimg, s.qscale, s.sp, xbar, c.status);
            FM_CK_LAUNCH();
            return FM_OK;
        }));
    }
    return FM_OK;
}

}  // namespace

template <typename T>
static fm_status ha_alloc(Ctx &c, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (hour-angle path)", __FILE__, __LINE__);
    c.allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return FM_OK;
}

// Geometry test, fringe groups, work partition and the per-handle phasor table.  The
// path is used for the tensor-core precisions when the LSTs are equally spaced by
// k = 1 .. 32 RA pixels, n_ant <= 64, n_lst <= 64, n_ra <= 512 and the buffers take at most half of
// the free device memory; otherwise c.ha.on stays false and the antenna form runs.
// CTAs contributing to each (M-tile, channel) segment when the forward's Q work units are cut
// into G contiguous ranges; sets s.grid and s.J (the most contributors of any segment)
static void ha_partition(Ctx &c, int G, std::vector<int> &ncontrib)
{
    HaState &s = c.ha;
    const int nchunk = c.D * s.nbc;
    const long long Q = (long long)s.nmt * c.F * nchunk;
    if (G > Q) G = (int)Q;
    if (G < 1) G = 1;
    s.grid = G;
    ncontrib.assign((size_t)s.nmt * c.F, 0);
    s.J = 1;
    for (size_t seg = 0; seg < ncontrib.size(); ++seg) {
        const int g0 = cta_of((long long)seg * nchunk, Q, G), g1 = cta_of((long long)(seg + 1) * nchunk - 1, Q, G);
        ncontrib[seg] = g1 - g0 + 1;
        if (ncontrib[seg] > s.J) s.J = ncontrib[seg];
    }
}

// Launch grids of the hour-angle contraction kernels (the autotuner's knobs): ctas_fwd for the
// forward (its unit partition is recomputed; 0 = one CTA per SM), ctas_adj for the adjoint
// (0 = one CTA per SM).  The partial-sum buffer holds the default grid's contributors, and a
// smaller grid never has more; a larger one is rejected.
fm_status ha_set_grids(Ctx &c, int ctas_fwd, int ctas_adj)
{
    HaState &s = c.ha;
    if (!s.on) { set_error("the handle does not run the hour-angle form"); return FM_ERR_UNSUPPORTED; }
    const int sm = sm_count();
    if (ctas_fwd < 0 || ctas_adj < 0 || ctas_fwd > sm || ctas_adj > sm) {
        set_error("launch grids must be in [0, %d] CTAs (0: one per SM)", sm);
        return FM_ERR_INVALID_ARG;
    }
    std::vector<int> ncontrib;
    const int Jmax = s.J_alloc;
    ha_partition(c, ctas_fwd > 0 ? ctas_fwd : sm, ncontrib);
    if (s.J > Jmax) {                      // cannot happen for G <= the default; kept as a guard
        ha_partition(c, sm, ncontrib);
        set_error("forward grid needs %d partial sums per segment, %d allocated", s.J, Jmax);
        return FM_ERR_INVALID_ARG;
    }
    s.J = Jmax;                            // the buffer's stride stays that of the allocation
    FM_CK(cudaMemcpy(s.ncontrib, ncontrib.data(), sizeof(int) * ncontrib.size(), cudaMemcpyHostToDevice));
    s.grid_adj = ctas_adj;
    return FM_OK;
}

fm_status ha_setup(Ctx &c)
{
    HaState &s = c.ha;
    s.on = false;
    if (c.prec < FM_PREC_BF16X1) return FM_OK;
    if (const char *e = getenv("FM_HA"))
        if (atoi(e) == 0) return FM_OK;
    if (c.A < 2 || c.R > 512) return FM_OK;
    const double dra = (c.cfg.ra_max - c.cfg.ra_min) / c.R;
    // LST step = k / q RA pixels (q <= 4): hour-angle cells of 1 / q pixel, k cells per LST
    int k = 1, q = 1;
    if (c.T > 1) {
        const double dl = c.lst[1] - c.lst[0];
        for (int t = 1; t < c.T; ++t)
            if (std::fabs(c.lst[t] - c.lst[0] - t * dl) > 1e-9 * dra) return FM_OK;
        const double kr = dl / dra;
        bool found = false;
        for (q = 1; q <= 4 && !found; ++q) {
            k = (int)std::llround(kr * q);
            if (k >= 1 && k <= 32 && std::fabs(kr * q - k) <= 1e-9 * k) found = true;
        }
        --q;
        if (!found) return FM_OK;
    }
    s.k = k;
    s.q = q;
    s.nh = (c.R - 1) * q + (c.T - 1) * k + 1;
    s.nhp = (s.nh + 127) / 128 * 128;
    s.nbc = s.nhp / 64;
    const int tc = c.T < HA_TCHUNK ? c.T : HA_TCHUNK;       // LSTs per pass
    s.npad = (tc + 15) / 16 * 16;
    if (s.npad < 16) s.npad = 16;
    // forward image: chunks j < Jc of 8 cells; the sky strip holds the Ly >= 8 Jc + 7 k + 8
    // elements the image reads (a multiple of 8, so strips stay 16-byte aligned)
    s.Jc = 8 * s.nbc + (s.npad / 8 - 1) * k;
    s.Lyc = 8 * s.Jc + 8 * k + 8;
    s.Ly = s.Lyc + ((c.T - 1) / HA_TCHUNK) * HA_TCHUNK * k;   // later passes start t0 k further in

    // fringe groups: equal baseline vectors (to 1 nm) up to sign
    bool group = true;
    if (const char *e = getenv("FM_HA_GROUPS"))
        if (atoi(e) == 0) group = false;
    std::vector<int> rep_i, rep_j, bmap(c.B), bi(c.B), bj(c.B);
    std::vector<double> rep_b;
    std::vector<std::vector<int>> members;
    for (int i = 0, b = 0; i < c.A; ++i)
        for (int j = i + 1; j < c.A; ++j, ++b) {
            bi[b] = i;
            bj[b] = j;
            const double v0 = c.ant[3 * i] - c.ant[3 * j], v1 = c.ant[3 * i + 1] - c.ant[3 * j + 1],
                         v2 = c.ant[3 * i + 2] - c.ant[3 * j + 2];
            int found = -1, cj = 0;
            if (group)
                for (size_t u = 0; u < rep_i.size() && found < 0; ++u) {
                    const double *r = &rep_b[3 * u];
                    const double dp = std::fmax(std::fabs(v0 - r[0]), std::fmax(std::fabs(v1 - r[1]), std::fabs(v2 - r[2])));
                    const double dm = std::fmax(std::fabs(v0 + r[0]), std::fmax(std::fabs(v1 + r[1]), std::fabs(v2 + r[2])));
                    if (dp < 1e-9) { found = (int)u; cj = 0; }
                    else if (dm < 1e-9) { found = (int)u; cj = 1; }
                }
            if (found < 0) {
                found = (int)rep_i.size();
                rep_i.push_back(i);
                rep_j.push_back(j);
                rep_b.push_back(v0);
                rep_b.push_back(v1);
                rep_b.push_back(v2);
                members.emplace_back();
            }
            bmap[b] = 2 * found + cj;
            members[found].push_back(2 * b + cj);
        }
    s.U = (int)rep_i.size();
    s.nmt = (s.U + 63) / 64;
    s.nkq = (s.U + 31) / 32;

    // Antennas whose phasors the table holds: a small set S such that every group has a
    // member pair inside S (greedy: add the antenna that completes the most groups, ties
    // broken by partial coverage); each group's representative is then such a pair.
    std::vector<int> in_s(c.A, 0), uncovered(s.U, 1);
    int n_unc = s.U;
    if (!group) {
        for (int a = 0; a < c.A; ++a) in_s[a] = 1;
        n_unc = 0;
    }
    while (n_unc > 0) {
        int best = -1;
        long long bfull = -1, bpart = -1;
        for (int a = 0; a < c.A; ++a) {
            if (in_s[a]) continue;
            long long full = 0, part = 0;
            for (int u = 0; u < s.U; ++u) {
                if (!uncovered[u]) continue;
                bool f1 = false, p1 = false;
                for (int m : members[u]) {
                    const int b = m >> 1, i = bi[b], j = bj[b];
                    const bool hi = in_s[i] || i == a, hj = in_s[j] || j == a;
                    if (hi && hj) { f1 = true; break; }
                    if (hi || hj) p1 = true;
                }
                full += f1;
                part += p1;
            }
            if (full > bfull || (full == bfull && part > bpart)) { best = a; bfull = full; bpart = part; }
        }
        in_s[best] = 1;
        for (int u = 0; u < s.U; ++u) {
            if (!uncovered[u]) continue;
            for (int m : members[u]) {
                const int b = m >> 1;
                if (in_s[bi[b]] && in_s[bj[b]]) { uncovered[u] = 0; --n_unc; break; }
            }
        }
    }
    std::vector<int> pos(c.A, -1);
    // the table holds at most 63 antennas plus its zero entry
    int n_in = 0;
    for (int a = 0; a < c.A; ++a) n_in += in_s[a] ? 1 : 0;
    if (n_in > 63) return FM_OK;
    s.nant = 0;
    for (int a = 0; a < c.A; ++a)
        if (in_s[a]) { pos[a] = s.nant; s.ant_of[s.nant] = a; ++s.nant; }
    // representatives inside S, member orientation relative to them
    for (int u = 0; u < s.U; ++u) {
        int rb = -1;
        for (int m : members[u]) {
            const int b = m >> 1;
            if (in_s[bi[b]] && in_s[bj[b]]) { rb = m; break; }
        }
        const int rflip = rb & 1;   // representative reversed w.r.t. the group's first member
        rep_i[u] = pos[bi[rb >> 1]];
        rep_j[u] = pos[bj[rb >> 1]];
        for (int &m : members[u]) m ^= rflip;
    }
    for (int u = 0; u < s.U; ++u)
        for (int m : members[u]) bmap[m >> 1] = 2 * u + (m & 1);

    // partition of the forward work units over the CTAs (the default grid: one CTA per SM;
    // the partial-sum buffer is sized for it, and a smaller grid needs no more contributors)
    std::vector<int> ncontrib;
    ha_partition(c, sm_count(), ncontrib);

    // both kernels' tiles must fit in shared memory
    {
        HaLayout L1, L2;
        const bool x3 = x3_of(c.prec);
        if (!make_layout_fwd(c, x3, L1) || !make_layout_adj(c, x3, L2)) return FM_OK;
    }

    // device memory, all of it within half of what is free
    const size_t e_n = (size_t)c.F * c.D * s.nbc * (s.nant + 1) * HA_EW;
    const size_t ys_n = 2 * (size_t)c.F * c.D * s.Ly;
    const size_t vp_n = (size_t)s.nmt * c.F * s.J * 128 * s.npad;
    const size_t q_n = (size_t)c.F * c.T * s.U * 2;
    const size_t qi_n = (size_t)c.F * s.nkq * 2 * s.npad * 128;
    const size_t need = 2 * e_n * 8 + ys_n * 2 + vp_n * 4 + q_n * 4 + qi_n + (size_t)c.B * 16 + (size_t)s.nmt * 64 * 8;
    size_t fr = 0, tot = 0;
    FM_CK(cudaMemGetInfo(&fr, &tot));
    if (need > fr / 2) return FM_OK;

    FM_TRY(ha_alloc(c, &s.E, e_n));
    FM_TRY(ha_alloc(c, &s.Ea, e_n));
    FM_TRY(ha_alloc(c, &s.uij, (size_t)s.nmt * 64));
    FM_TRY(ha_alloc(c, &s.bmap, (size_t)c.B));
    FM_TRY(ha_alloc(c, &s.moff, (size_t)s.U + 1));
    FM_TRY(ha_alloc(c, &s.mem, (size_t)c.B));
    FM_TRY(ha_alloc(c, &s.ncontrib, ncontrib.size()));
    FM_TRY(ha_alloc(c, &s.ys, ys_n));
    FM_CK(cudaMemset(s.ys, 0, ys_n * sizeof(uint16_t)));     // strip elements outside the pixels stay zero
    FM_TRY(ha_alloc(c, &s.xmax, (size_t)c.F));
    FM_TRY(ha_alloc(c, &s.vpart, vp_n));
    s.J_alloc = s.J;
    FM_TRY(ha_alloc(c, &s.q32, q_n));
    FM_TRY(ha_alloc(c, &s.qmax_ft, (size_t)c.F * c.T));
    FM_TRY(ha_alloc(c, &s.qscale, (size_t)c.F));
    FM_TRY(ha_alloc(c, &s.qimg, qi_n));

    std::vector<int2> huij((size_t)s.nmt * 64, make_int2(s.nant, s.nant));   // padding: the zero entry
    for (int u = 0; u < s.U; ++u) huij[u] = make_int2(rep_i[u], rep_j[u]);
    s.rep_ant.assign(2 * (size_t)s.U, 0);
    for (int u = 0; u < s.U; ++u) {
        s.rep_ant[2 * u] = s.ant_of[rep_i[u]];
        s.rep_ant[2 * u + 1] = s.ant_of[rep_j[u]];
    }
    std::vector<int> hoff(s.U + 1, 0), hmem;
    hmem.reserve(c.B);
    for (int u = 0; u < s.U; ++u) {
        hoff[u] = (int)hmem.size();
        for (int m : members[u]) hmem.push_back(m);
    }
    hoff[s.U] = (int)hmem.size();
    FM_CK(cudaMemcpy(s.uij, huij.data(), sizeof(int2) * huij.size(), cudaMemcpyHostToDevice));
    FM_CK(cudaMemcpy(s.bmap, bmap.data(), sizeof(int) * bmap.size(), cudaMemcpyHostToDevice));
    FM_CK(cudaMemcpy(s.moff, hoff.data(), sizeof(int) * hoff.size(), cudaMemcpyHostToDevice));
    FM_CK(cudaMemcpy(s.mem, hmem.data(), sizeof(int) * hmem.size(), cudaMemcpyHostToDevice));
    FM_CK(cudaMemcpy(s.ncontrib, ncontrib.data(), sizeof(int) * ncontrib.size(), cudaMemcpyHostToDevice));

    // response scale 2^e, e even, with 2^e dOmega_max <= 2^14 (the beam is at most 1)
    int e2 = 0;
    if (c.domega_max > 0.f) {
        e2 = (int)std::floor(std::log2(16384.0 / (double)c.domega_max));
        if (e2 & 1) --e2;
    }
    s.sp = (float)std::ldexp(1.0, e2);
    HaTabArgs a;
    a.F = c.F; a.D = c.D; a.R = c.R; a.A = s.nant + 1; a.A_all = c.A; a.nh = s.nh; a.nhp = s.nhp; a.nbc = s.nbc;
    a.q = s.q;
    for (int q = 0; q < s.nant; ++q) a.ant[q] = s.ant_of[q];
    a.lst0 = c.lst[0]; a.ra_min = c.cfg.ra_min; a.dra = dra;
    a.dec_min = c.cfg.dec_min; a.ddec = (c.cfg.dec_max - c.cfg.dec_min) / c.D;
    a.lat = c.cfg.latitude_rad; a.amp_scale = std::ldexp(1.0, e2 / 2);
    a.kap64 = c.g.kap64; a.bcoef64 = c.g.bcoef64; a.domega64 = c.g.domega64;
    a.airy = c.g.beam32 != nullptr; a.dew = c.g.dish_ew; a.dns = c.g.dish_ns; a.freq = c.g.freq64;
    s.lst0 = c.lst[0];
    s.dra = dra;
    k_ha_table<<<2048, 256>>>(a, 1, reinterpret_cast<float *>(s.E));
    FM_CK_LAUNCH();
    k_ha_table<<<2048, 256>>>(a, 0, reinterpret_cast<float *>(s.Ea));
    FM_CK_LAUNCH();
    FM_CK(cudaDeviceSynchronize());
    s.on = true;
    return FM_OK;
}

// U[f][t][b] = V_b(1) in FP64 through the hour-angle geometry (k_ha_monopole); returns
// FM_ERR_UNSUPPORTED when the cells or LSTs exceed its shared memory (the caller then uses
// the direct FP64 sum)
fm_status ha_monopole(Ctx &c, float *U, cudaStream_t st)
{
    const HaState &s = c.ha;
    if (!s.on) return FM_ERR_UNSUPPORTED;
    const size_t smem = sizeof(double) * 2 * ((size_t)s.nh + c.T);
    if (smem > 200 * 1024) return FM_ERR_UNSUPPORTED;
    int *rep = nullptr;
    FM_CK(cudaMalloc(&rep, sizeof(int) * s.rep_ant.size()));
    cudaError_t e = cudaMemcpy(rep, s.rep_ant.data(), sizeof(int) * s.rep_ant.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(rep);
        return cuda_fail(e, "cudaMemcpy (monopole groups)", __FILE__, __LINE__);
    }
    HaMonoArgs a;
    a.F = c.F; a.D = c.D; a.R = c.R; a.T = c.T; a.B = c.B; a.U = s.U; a.k = s.k; a.q = s.q; a.nh = s.nh;
    a.A_all = c.A;
    a.lst0 = s.lst0; a.ra_min = c.cfg.ra_min; a.dra = s.dra;
    a.dec_min = c.cfg.dec_min; a.ddec = (c.cfg.dec_max - c.cfg.dec_min) / c.D; a.lat = c.cfg.latitude_rad;
    a.kap64 = c.g.kap64; a.bcoef64 = c.g.bcoef64; a.domega64 = c.g.domega64;
    a.airy = c.g.beam32 != nullptr; a.dew = c.g.dish_ew; a.dns = c.g.dish_ns; a.freq = c.g.freq64;
    a.rep = rep; a.moff = s.moff; a.mem = s.mem;
    a.ug = nullptr;
    fm_status rc = FM_OK;
    if (!c.ha.ug) {
        void *q = nullptr;
        if ((e = cudaMalloc(&q, sizeof(float) * 2 * (size_t)c.F * c.T * s.U)) != cudaSuccess) {
            cudaFree(rep);
            return cuda_fail(e, "cudaMalloc (group monopoles)", __FILE__, __LINE__);
        }
        c.allocs.push_back(q);
        c.ha.ug = reinterpret_cast<float *>(q);
    }
    a.ug = c.ha.ug;
    if ((e = smem_opt_in(k_ha_monopole)) != cudaSuccess) rc = cuda_fail(e, "smem_opt_in", __FILE__, __LINE__);
    if (rc == FM_OK) {
        k_ha_monopole<<<(unsigned)((long long)c.F * s.U), 256, smem, st>>>(a, U);
        __atomic_fetch_add(&g_launches, 1LL, __ATOMIC_RELAXED);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e, "k_ha_monopole", __FILE__, __LINE__);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess && rc == FM_OK) rc = cuda_fail(e, "monopole", __FILE__, __LINE__);
    cudaFree(rep);
    return rc;
}

fm_status launch_vis_ha(Ctx &c, const float *x, float *vis, cudaStream_t st, const float *dc, long long dcs,
                        bool xmax_ready, bool strips_ready, bool partials_only)
{
    const HaDev h = make_dev(c);
    const bool x3 = x3_of(c.prec), po = partials_only;
    if (f16_of(c.prec))
        return x3 ? vis_ha_launch<1, true>(c, h, x, vis, st, dc, dcs, xmax_ready, strips_ready, po)
                  : vis_ha_launch<1, false>(c, h, x, vis, st, dc, dcs, xmax_ready, strips_ready, po);
    return x3 ? vis_ha_launch<0, true>(c, h, x, vis, st, dc, dcs, xmax_ready, strips_ready, po)
              : vis_ha_launch<0, false>(c, h, x, vis, st, dc, dcs, xmax_ready, strips_ready, po);
}

bool ha_vsrc(const Ctx &c, const float *dc, long long dcs, HaVSrc &v)
{
    const HaState &s = c.ha;
    if (!s.on || c.T > HA_TCHUNK || (dc && !s.ug)) return false;
    if (const char *e = getenv("FM_HA_FUSED_CHI2"))      // 0: V finished by its own kernel
        if (atoi(e) == 0) return false;
    v.vpart = s.vpart;
    v.ncontrib = s.ncontrib;
    v.bmap = s.bmap;
    v.xmax = s.xmax;
    v.dc = dc;
    v.dcs = dcs;
    v.ug = s.ug;
    v.sp = s.sp;
    v.J = s.J;
    v.npad = s.npad;
    v.nmt = s.nmt;
    v.F = c.F;
    return true;
}

bool ha_strip_args(const Ctx &c, StripArgs &sa)
{
    if (!c.ha.on || c.D > 128) return false;
    if (const char *e = getenv("FM_MODES_STRIPS"))      // 0: strips from their own kernel
        if (atoi(e) == 0) return false;
    const HaState &s = c.ha;
    sa.hi = s.ys;
    sa.lo = s.ys + (size_t)c.F * c.D * s.Ly;
    sa.Ly = s.Ly;
    sa.q = s.q;
    sa.off = s.nhp - 1 - (c.R - 1) * s.q;       // element of pixel 0 (k_ha_yprep)
    sa.bf16 = f16_of(c.prec) ? 0 : 1;
    return true;
}

fm_status launch_adjoint_ha(Ctx &c, const float *omega, float *xbar, cudaStream_t st, bool q_ready)
{
    const HaDev h = make_dev(c);
    const bool x3 = x3_of(c.prec);
    if (f16_of(c.prec))
        return x3 ? adj_ha_launch<1, true>(c, h, omega, xbar, st, q_ready)
                  : adj_ha_launch<1, false>(c, h, omega, xbar, st, q_ready);
    return x3 ? adj_ha_launch<0, true>(c, h, omega, xbar, st, q_ready)
              : adj_ha_launch<0, false>(c, h, omega, xbar, st, q_ready);
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_set_launch_grids(fm_handle h, int ctas_fwd, int ctas_adj)
{
    if (!h) {
        set_error("invalid argument: handle is NULL");
        return FM_ERR_INVALID_ARG;
    }
    return ha_set_grids(*reinterpret_cast<Ctx *>(h), ctas_fwd, ctas_adj);
}

extern "C" fm_status fm_get_launch_grids(fm_handle h, int32_t *out)
{
    if (!h || !out) {
        set_error("invalid argument: handle and out are required");
        return FM_ERR_INVALID_ARG;
    }
    const Ctx &c = *reinterpret_cast<const Ctx *>(h);
    out[0] = c.ha.on ? c.ha.grid : 0;
    out[1] = c.ha.on ? (c.ha.grid_adj > 0 ? c.ha.grid_adj : (sm_count() < c.F * c.D ? sm_count() : c.F * c.D)) : 0;
    return FM_OK;
}
