// Tensor-core (tcgen05, sm_103a) fringe contraction and its adjoint.
//
// Forward (Eq. rime_discrete with K_pq = E_p conj(E_q), b_pq = r_p - r_q):
//   for each (channel, LST) task, D = Ahat W Ahat^T with Ahat the real [2 n_ant x n_pix]
//   matrix whose rows 2i, 2i+1 are Re E_i, Im E_i (E_i = exp(-2 pi i nu r_i.s/c)) and
//   W = diag(dOmega A x).  Then V_ij = D[2i][2j] + D[2i+1][2j+1] + i (D[2i+1][2j] - D[2i][2j+1]).
//   The MMA reads A_op = Ahat W (M = 128 rows, zero beyond 2 n_ant) and B_op = Ahat
//   (N = 2 n_ant rounded up to 16) from shared memory in the 128-byte-swizzled K-major
//   layout, 64 pixels (one swizzle row) per pipeline stage; the accumulator lives in
//   TMEM.  Operands are generated in the kernel (never stored in HBM): two-float phase
//   in turns, sincos, then BF16 hi/lo split.  BF16x3 adds hi*lo + lo*hi products.
//
// Adjoint: for each (channel, tile of 128 pixels), looping over LSTs,
//   D[p][n] = sum_k Ehat^T[p][k] Chat[n][k] with Ehat^T rows = pixels and interleaved
//   (Re E_j, Im E_j) along K, Chat the real form of the Hermitian residual-weight matrix
//   C (C_ij = omega_ij for i < j, conj(omega_ji) for i > j): D[p][2i] + i D[p][2i+1] =
//   Y_i(p) = sum_j C_ij E_j(p), and xbar_p += dOmega A sum_i Re(conj(E_i) Y_i) / 2.
//
// Synchronisation: one mbarrier per stage, completed by tcgen05.commit after the MMAs
// reading that stage; every wait is bounded by a clock limit, after which the kernel
// records FM_ERR_TIMEOUT, drains its own MMAs (bounded), frees TMEM and returns.
#include <cstdlib>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fm_internal.cuh"
#include "tc_ptx.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int KST = 64;                               // pixels per stage (one swizzle row of bf16)
template <int NC = 3>
__device__ __forceinline__ float phase_frac(const float *kap, const float *s)
{
    float accf = 0.f, acce = 0.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
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

// sin and cos of 2 pi r for r in [-1/2, 1/2] turns: quadrant reduction q = rint(4 r)
// (r - q/4 is exact), y = 2 pi (r - q/4) in [-pi/4, pi/4], Taylor series of sin and cos
// to degree 9 and 10 (truncation below 2e-9 there), then rotation by q quarter turns.
__device__ __forceinline__ void sincos_turns(float r, float &s, float &c)
{
    const float q = rintf(4.f * r);
    const float y = (r - 0.25f * q) * 6.28318530717958647692f;
    const float y2 = y * y;
    const float sp = fmaf(y * y2, fmaf(y2, fmaf(y2, fmaf(y2, 2.7557319e-6f, -1.9841270e-4f), 8.3333333e-3f),
                                       -1.6666667e-1f), y);
    const float cp = fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, -2.7557319e-7f, 2.4801587e-5f), -1.3888889e-3f),
                                            4.1666667e-2f), -0.5f), 1.f);
    const int qi = ((int)q) & 3;
    s = (qi == 0) ? sp : (qi == 1) ? cp : (qi == 2) ? -sp : -cp;
    c = (qi == 0) ? cp : (qi == 1) ? -sp : (qi == 2) ? -cp : sp;
}

// E = exp(-2 pi i frac); FAST uses the hardware approximation (abs. error ~4e-7), for
// the single-product modes whose 2^-9 / 2^-12 operand rounding dominates anyway
template <bool FAST = false>
__device__ __forceinline__ void phasor_of(float fr, float &er, float &ei)
{
    float sn, cs;
    if (FAST) __sincosf(6.28318530717958647692f * fr, &sn, &cs);
    else sincos_turns(fr, sn, cs);
    er = cs;
    ei = -sn;
}

// exp(-2 pi i d) for a small phase d (|d| <= 1/8 turn, the channel-step factor of the
// frequency recurrence): Taylor series of sin and cos to degree 9 / 10 in y = 2 pi d,
// no quadrant reduction needed (truncation below 2e-9 for |y| <= pi/4)
__device__ __forceinline__ void phasor_small(float d, float &er, float &ei)
{
    const float y = d * 6.28318530717958647692f;
    const float y2 = y * y;
    const float sp = fmaf(y * y2, fmaf(y2, fmaf(y2, fmaf(y2, 2.7557319e-6f, -1.9841270e-4f), 8.3333333e-3f),
                                       -1.6666667e-1f), y);
    const float cp = fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, -2.7557319e-7f, 2.4801587e-5f), -1.3888889e-3f),
                                            4.1666667e-2f), -0.5f), 1.f);
    er = cp;
    ei = -sp;
}

__device__ __forceinline__ float pixel_w(const DevGeom &g, int f, int t, int p)
{
    if (g.beam32) return g.domega32[p / g.R] * g.beam32[((size_t)f * g.T + t) * g.npix + p];
    float z2 = g.za2_32[(size_t)t * g.npix + p];
    if (z2 < 0.f) return 0.f;
    return g.domega32[p / g.R] * __expf(g.bcoef32[f] * z2);
}

__device__ __forceinline__ void load_s6(const DevGeom &g, int t, int p, float *s)
{
    const float4 *q = reinterpret_cast<const float4 *>(g.s32 + ((size_t)t * g.npix + p) * 6);
    // 6 floats at a 24-byte stride: read as float2 x 3 (8-byte aligned)
    const float2 *q2 = reinterpret_cast<const float2 *>(q);
    float2 a = q2[0], b = q2[1], c = q2[2];
    s[0] = a.x; s[1] = a.y; s[2] = b.x; s[3] = b.y; s[4] = c.x; s[5] = c.y;
}

__device__ __forceinline__ int pair_idx(int i, int j, int A) { return i * A - (i * (i + 1)) / 2 + (j - i - 1); }

struct FwdLayout {
    int npad, nstage, ncols;
    uint32_t a_bytes, b_bytes, stage_bytes;
};

// max |x[f][p]| * dOmega_max -> power-of-two scale putting the largest A-operand value
// below 2^14 (FP16 range), one CTA per channel
__global__ void __launch_bounds__(256) k_chan_scale(int npix, const float *__restrict__ x, float domega_max,
                                                   float *__restrict__ scale)
{
    __shared__ float red[256];
    const int f = blockIdx.x;
    float m = 0.f;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) m = fmaxf(m, fabsf(x[(size_t)f * npix + p]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float mm = red[0] * domega_max;
        float sc = 1.f;
        if (mm > 0.f && isfinite(mm)) {
            int e;
            frexpf(mm, &e);                // mm < 2^e
            sc = ldexpf(1.f, 14 - e);
        }
        scale[f] = sc;
    }
}

// ------------------------------------------------------------------ forward kernel
// Producers: lane l of every warp owns pixels 2l, 2l+1 of the 64-pixel stage; warp w
// generates antennas w, w+8, ...  Each thread writes 32-bit words (2 pixels) of rows
// 2i (Re) and 2i+1 (Im) of A_op = W Ahat and B_op = Ahat, hi and (x3) lo parts.
// Warp-specialised forward: warps 0-15 produce operand stages, warp 20 (one lane) issues
// the MMAs, warps 16-19 drain the TMEM accumulators.  Hand-offs use mbarriers only:
//   full[s]     16 producer-warp arrivals -> stage s holds operands
//   empty[s]    tcgen05.commit after the MMAs that read stage s
//   accfull[q]  tcgen05.commit after the last MMA of a pixel sub-range into set q
//   accempty[q] 4 epilogue-warp arrivals after set q was read
// Stage order (all roles enumerate it identically): task -> 64-pixel chunk j -> channel r
// of the task's frequency-recurrence group.  Accumulator set q = sub-range parity, so
// the epilogue of one sub-range overlaps the MMAs of the next; partial visibilities
// are summed in FP32 in shared memory and written once per task.
constexpr int FWD_PROD_WARPS = 16;
constexpr int FWD_MMA_WARP = 20;
constexpr int FWD_THREADS = 21 * 32;

template <int ET, bool X3, int KMAX>
__global__ void __launch_bounds__(FWD_THREADS, 1)
k_vis_tc(DevGeom g, FwdLayout L, int rch, int sub, const float *__restrict__ x, const float *__restrict__ chan_scale,
         float *__restrict__ vis)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t stages_bytes = (uint32_t)L.nstage * L.stage_bytes;
    float *vpart = reinterpret_cast<float *>(gbase + stages_bytes);            // [rch][B][2]
    const uint32_t bar_off = stages_bytes + (uint32_t)(rch * g.B * 2 * 4 + 15) / 16 * 16;
    const uint32_t full0 = base + bar_off, empty0 = full0 + 8 * L.nstage;
    const uint32_t accf0 = empty0 + 8 * L.nstage, acce0 = accf0 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + bar_off + 16 * L.nstage + 32);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + bar_off + 16 * L.nstage + 36);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows_used = 2 * g.A;
    const int ntl = X3 ? 2 : 1;
    for (int s = 0; s < L.nstage; ++s) {            // zero the padding rows once
        uint8_t *st = gbase + (size_t)s * L.stage_bytes;
        for (int tl = 0; tl < ntl; ++tl) {
            uint8_t *ta = st + tl * L.a_bytes;
            for (int e = tid; e < (128 - rows_used) * 8; e += FWD_THREADS)
                reinterpret_cast<uint4 *>(ta + (size_t)(rows_used + e / 8) * 128)[e % 8] = make_uint4(0, 0, 0, 0);
            uint8_t *tb = st + ntl * L.a_bytes + tl * L.b_bytes;
            for (int e = tid; e < (L.npad - rows_used) * 8; e += FWD_THREADS)
                reinterpret_cast<uint4 *>(tb + (size_t)(rows_used + e / 8) * 128)[e % 8] = make_uint4(0, 0, 0, 0);
        }
    }
    if (tid == 0) {
        for (int s = 0; s < L.nstage; ++s) {
            mbar_init(full0 + 8 * s, FWD_PROD_WARPS);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(accf0 + 8 * q, 1);
            mbar_init(acce0 + 8 * q, 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == FWD_MMA_WARP) tmem_alloc(su32(tmem_slot), (uint32_t)L.ncols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;
    const int nst = (g.npix + KST - 1) / KST;
    const int ngrp = (g.F + rch - 1) / rch;
    const int ntask = ngrp * g.T;
    const int set_cols = rch * L.npad;

    if (warp < FWD_PROD_WARPS) {
        // ------------------------------------------------------------ producers
        const uint32_t wsub = (uint32_t)(lane & 3) * 4u;
        const int wchunk = lane >> 2;
        int s = 0;                 // ring slot of the next stage
        uint32_t phase = 0;        // its fill count parity
        bool wrapped = false;      // the slot was filled before (wait for its release)
        for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
            const int t = task % g.T, f0 = (task / g.T) * rch;
            const int nr = min(rch, g.F - f0);
            for (int j = 0; j < nst; ++j) {
                const int pa = j * KST + 2 * lane, pb = pa + 1;
                const bool va = pa < g.npix, vb = pb < g.npix;
                float sa[6], sb[6], za = -1.f, zb = -1.f, da = 0.f, db = 0.f;
                if (va) { load_s6(g, t, pa, sa); za = g.za2_32[(size_t)t * g.npix + pa]; da = g.dompix32[pa]; }
                if (vb) { load_s6(g, t, pb, sb); zb = g.za2_32[(size_t)t * g.npix + pb]; db = g.dompix32[pb]; }
                float er[KMAX][2], ei[KMAX][2], dr[KMAX][2], di[KMAX][2];
                for (int r = 0; r < nr; ++r) {
                    const int f = f0 + r;
                    const float scale = ET == 1 ? chan_scale[f] : 1.f;
                    const float bc = g.bcoef32[f];
                    const float *bt = g.beam32 ? g.beam32 + ((size_t)f * g.T + t) * g.npix : nullptr;
                    const float ba = bt ? (va ? bt[pa] : 0.f) : ((za >= 0.f) ? __expf(bc * za) : 0.f);
                    const float bb = bt ? (vb ? bt[pb] : 0.f) : ((zb >= 0.f) ? __expf(bc * zb) : 0.f);
                    const float wa = va ? da * ba * x[(size_t)f * g.npix + pa] * scale : 0.f;
                    const float wb = vb ? db * bb * x[(size_t)f * g.npix + pb] * scale : 0.f;
#pragma unroll
                    for (int k = 0; k < KMAX; ++k) {
                        const int i = warp + FWD_PROD_WARPS * k;
                        if (i >= g.A) continue;
                        if (r == 0) {
                            float k6[6];
#pragma unroll
                            for (int q = 0; q < 6; ++q) k6[q] = g.kap32[((size_t)f * g.A + i) * 6 + q];
                            er[k][0] = ei[k][0] = er[k][1] = ei[k][1] = 0.f;
                            const float d0 = g.dkap32[3 * i], d1 = g.dkap32[3 * i + 1], d2 = g.dkap32[3 * i + 2];
                            if (g.flat_array) {
                                if (va) phasor_of<!X3>(phase_frac<2>(k6, sa), er[k][0], ei[k][0]);
                                if (vb) phasor_of<!X3>(phase_frac<2>(k6, sb), er[k][1], ei[k][1]);
                                if (nr > 1) {
                                    phasor_small(d0 * sa[0] + d1 * sa[2], dr[k][0], di[k][0]);
                                    phasor_small(d0 * sb[0] + d1 * sb[2], dr[k][1], di[k][1]);
                                }
                            } else {
                                if (va) phasor_of<!X3>(phase_frac<3>(k6, sa), er[k][0], ei[k][0]);
                                if (vb) phasor_of<!X3>(phase_frac<3>(k6, sb), er[k][1], ei[k][1]);
                                if (nr > 1) {
                                    phasor_small(d0 * sa[0] + d1 * sa[2] + d2 * sa[4], dr[k][0], di[k][0]);
                                    phasor_small(d0 * sb[0] + d1 * sb[2] + d2 * sb[4], dr[k][1], di[k][1]);
                                }
                            }
                        } else {
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const float a = er[k][u], b = ei[k][u];
                                er[k][u] = a * dr[k][u] - b * di[k][u];
                                ei[k][u] = a * di[k][u] + b * dr[k][u];
                            }
                        }
                    }
                    bool ok = true;
                    if (lane == 0 && wrapped) ok = mbar_wait_ab(empty0 + 8 * s, phase ^ 1u, abort_flag);
                    __syncwarp();
                    if (*abort_flag || !ok) goto done;
                    {
                        uint8_t *st = gbase + (size_t)s * L.stage_bytes;
                        uint8_t *a_hi = st, *a_lo = st + L.a_bytes;
                        uint8_t *b_hi = st + ntl * L.a_bytes, *b_lo = b_hi + L.b_bytes;
#pragma unroll
                        for (int k = 0; k < KMAX; ++k) {
                            const int i = warp + FWD_PROD_WARPS * k;
                            if (i >= g.A) continue;
                            uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
                            Elem<ET>::split(wa * er[k][0], wb * er[k][1], h0, l0);
                            Elem<ET>::split(wa * ei[k][0], wb * ei[k][1], h1, l1);
                            Elem<ET>::split(er[k][0], er[k][1], h2, l2);
                            Elem<ET>::split(ei[k][0], ei[k][1], h3, l3);
                            const uint32_t ore = sw128_off(2 * i, wchunk) + wsub, oim = sw128_off(2 * i + 1, wchunk) + wsub;
                            *reinterpret_cast<uint32_t *>(a_hi + ore) = h0;
                            *reinterpret_cast<uint32_t *>(a_hi + oim) = h1;
                            *reinterpret_cast<uint32_t *>(b_hi + ore) = h2;
                            *reinterpret_cast<uint32_t *>(b_hi + oim) = h3;
                            if (X3) {
                                *reinterpret_cast<uint32_t *>(a_lo + ore) = l0;
                                *reinterpret_cast<uint32_t *>(a_lo + oim) = l1;
                                *reinterpret_cast<uint32_t *>(b_lo + ore) = l2;
                                *reinterpret_cast<uint32_t *>(b_lo + oim) = l3;
                            }
                        }
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full0 + 8 * s);
                    if (++s == L.nstage) { s = 0; phase ^= 1u; wrapped = true; }
                }
            }
        }
    } else if (warp == FWD_MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, L.npad, Elem<ET>::kFmt);
            long long sr = 0;
            int s = 0, last_s = -1;
            uint32_t phase = 0, last_phase = 0;
            for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
                const int f0 = (task / g.T) * rch;
                const int nr = min(rch, g.F - f0);
                int jmod = 0;              // j % sub
                for (int j = 0; j < nst; ++j) {
                    const int q = (int)(sr & 1);
                    if (jmod == 0 && (sr >> 1) >= 1) {
                        if (!mbar_wait_ab(acce0 + 8 * q, (uint32_t)(((sr >> 1) - 1) & 1), abort_flag)) goto mma_done;
                    }
                    for (int r = 0; r < nr; ++r) {
                        if (!mbar_wait_ab(full0 + 8 * s, phase, abort_flag)) goto mma_done;
                        tc_fence_after();
                        const uint32_t sa_hi = base + (uint32_t)s * L.stage_bytes;
                        const uint32_t sa_lo = sa_hi + L.a_bytes;
                        const uint32_t sb_hi = sa_hi + (uint32_t)ntl * L.a_bytes;
                        const uint32_t sb_lo = sb_hi + L.b_bytes;
                        const uint32_t dacc = tmem_d + (uint32_t)(q * set_cols + r * L.npad);
#pragma unroll
                        for (int kk = 0; kk < KST / 16; ++kk) {
                            const uint32_t off = 32u * kk;
                            const uint64_t dah = sdesc_sw128(sa_hi + off), dbh = sdesc_sw128(sb_hi + off);
                            mma_bf16(dacc, dah, dbh, idesc, (jmod > 0 || kk > 0) ? 1u : 0u);
                            if (X3) {
                                mma_bf16(dacc, dah, sdesc_sw128(sb_lo + off), idesc, 1u);
                                mma_bf16(dacc, sdesc_sw128(sa_lo + off), dbh, idesc, 1u);
                            }
                        }
                        mma_commit(empty0 + 8 * s);
                        last_s = s;
                        last_phase = phase;
                        if (++s == L.nstage) { s = 0; phase ^= 1u; }
                    }
                    if (jmod == sub - 1 || j == nst - 1) {
                        mma_commit(accf0 + 8 * q);
                        ++sr;
                    }
                    if (++jmod == sub) jmod = 0;
                }
            }
        mma_done:
            if (*abort_flag && last_s >= 0) {
                // drain this CTA's MMAs before TMEM is freed (bounded)
                long long t0 = clock64();
                while (clock64() - t0 < WAIT_CYCLES) {
                    uint32_t ok;
                    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                                 : "=r"(ok) : "r"(empty0 + 8 * last_s), "r"(last_phase) : "memory");
                    if (ok) break;
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 8-11)
        const int quarter = warp & 3;                   // TMEM lanes 32*quarter .. +31
        const int row = 32 * quarter + lane, i = row >> 1;
        const bool even = (row & 1) == 0;
        long long sr = 0;
        for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
            const int t = task % g.T, f0 = (task / g.T) * rch;
            const int nr = min(rch, g.F - f0);
            for (int j = sub - 1;; j += sub) {
                if (j >= nst) j = nst - 1;
                const int q = (int)(sr & 1);
                const bool first = j < sub, last_sub = j == nst - 1;
                bool ok = true;
                if (lane == 0) ok = mbar_wait_ab(accf0 + 8 * q, (uint32_t)((sr >> 1) & 1), abort_flag);
                __syncwarp();
                if (*abort_flag || !ok) goto done;
                tc_fence_after();
                for (int r = 0; r < nr; ++r) {
                    for (int c0 = 0; c0 < L.npad; c0 += 16) {
                        float v[16], pv[16];
                        tmem_ld16(tmem_d + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(q * set_cols + r * L.npad + c0), v);
#pragma unroll
                        for (int qq = 0; qq < 16; ++qq) pv[qq] = __shfl_xor_sync(0xffffffffu, v[qq], 1);
                        if (even && i < g.A) {
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) {
                                const int jn = c0 / 2 + jj;
                                if (jn > i && jn < g.A) {
                                    // each (channel, pair) has one owner thread: no synchronisation
                                    const int b = pair_idx(i, jn, g.A);
                                    float *o = vpart + ((size_t)r * g.B + b) * 2;
                                    float re = v[2 * jj] + pv[2 * jj + 1];
                                    float im = pv[2 * jj] - v[2 * jj + 1];
                                    if (!first) { re += o[0]; im += o[1]; }
                                    if (last_sub) {
                                        const float inv = ET == 1 ? 1.f / chan_scale[f0 + r] : 1.f;
                                        const size_t go = (((size_t)(f0 + r) * g.T + t) * g.B + b) * 2;
                                        vis[go] = re * inv;
                                        vis[go + 1] = im * inv;
                                    } else {
                                        o[0] = re;
                                        o[1] = im;
                                    }
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * q);
                ++sr;
                if (last_sub) break;
            }
        }
    }
done:
    __syncthreads();
    if (*abort_flag && tid == 0) atomicExch(g.status, (int)FM_ERR_TIMEOUT);
    if (warp == FWD_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem_d, (uint32_t)L.ncols);
    }
}

// ------------------------------------------------------------------ adjoint kernel
// One task per (channel, LST).  Warp-specialised like the forward:
//   producers (warps 0-15): per task, warp 0 stages omega and its FP16 scale (sready),
//     all build the residual-weight tile B = Chat (bfull); then 128-pixel chunks of
//     A = Ehat^T (rows = pixels, K = interleaved Re/Im phasors) go into a 2-slot ring;
//   MMA warp (20): D(s) = A(s) B^T into TMEM slot s, commits dfull[s] and empty[s], and
//     bempty once the task's last MMA has read B;
//   epilogue (warps 16-19): wbar_p = A_p dOmega sum_i Re(conj(E_i) Y_i) / 2 from D(s) and
//     the phasors still in A(s), then releases the slot (empty[s]: 1 commit + 4 warps).
// The pixel adjoint of each (channel, LST) goes to wbar[f][t][p]; k_wbar_reduce sums t.
struct AdjLayout {
    int npad, katoms, ksteps, ncols;
    uint32_t a_bytes, b_bytes;        // one hi (or lo) tile
    uint32_t abuf_bytes;              // A slot (hi + lo)
    uint32_t b_off;                   // offset of the B tiles (after the A slots)
    uint32_t om_off;                  // omega staging [2B] floats
    uint32_t meta_off;                // slot metadata, barriers, TMEM slot, abort flag
};
constexpr int ADJ_SLOTS = 2;
constexpr int ADJ_PROD_WARPS = 16;
constexpr int ADJ_MMA_WARP = 20;
constexpr int ADJ_THREADS = 21 * 32;

template <int ET, bool X3>
__global__ void __launch_bounds__(ADJ_THREADS, 1)
k_adj_tc(DevGeom g, AdjLayout L, const float *__restrict__ omega, float *__restrict__ wbar)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    float *som = reinterpret_cast<float *>(gbase + L.om_off);
    uint8_t *meta = gbase + L.meta_off;
    float *slot_scale = reinterpret_cast<float *>(meta);             // [2]
    int *slot_ft = reinterpret_cast<int *>(meta + 8);                // [2]
    int *slot_p0 = reinterpret_cast<int *>(meta + 16);               // [2]
    float *task_scale = reinterpret_cast<float *>(meta + 24);
    float *wmax = reinterpret_cast<float *>(meta + 32);              // unused slot (alignment)
    const uint32_t bar0 = base + L.meta_off + 64;
    const uint32_t full0 = bar0, empty0 = bar0 + 16, dfull0 = bar0 + 32;
    const uint32_t sready = bar0 + 48, bfull = bar0 + 56, bempty = bar0 + 64;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(meta + 64 + 72);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(meta + 64 + 76);
    (void)wmax;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kused = 2 * g.A;
    const uint32_t a_atom = 128u * 128u, b_atom = (uint32_t)L.npad * 128u;
    uint8_t *bt_hi = gbase + L.b_off, *bt_lo = bt_hi + L.b_bytes;

    for (uint32_t e = tid; e < L.om_off / 16; e += ADJ_THREADS)
        reinterpret_cast<uint4 *>(gbase)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int q = 0; q < ADJ_SLOTS; ++q) {
            mbar_init(full0 + 8 * q, ADJ_PROD_WARPS);
            mbar_init(empty0 + 8 * q, 1 + 4);
            mbar_init(dfull0 + 8 * q, 1);
        }
        mbar_init(sready, 1);
        mbar_init(bfull, ADJ_PROD_WARPS);
        mbar_init(bempty, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == ADJ_MMA_WARP) tmem_alloc(su32(tmem_slot), (uint32_t)L.ncols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem0 = *tmem_slot;
    const int nchk = (g.npix + 127) / 128;
    const int ntask = g.F * g.T;
    const int nchunk = (kused + 7) / 8;            // 16-byte chunks of K actually used

    if (warp < ADJ_PROD_WARPS) {
        // ------------------------------------------------------------ producers
        const int ptid = tid;                      // 0 .. 511
        // this thread's (pixel row, K chunk) items, the same for every chunk
        int it_row[3], it_kc[3], nits = 0;
        for (int item = ptid; item < 128 * nchunk && nits < 3; item += ADJ_PROD_WARPS * 32) {
            it_row[nits] = item / nchunk;
            it_kc[nits] = item % nchunk;
            ++nits;
        }
        long long gs = 0;
        int n = 0;
        for (int ft = blockIdx.x; ft < ntask; ft += gridDim.x, ++n) {
            const int f = ft / g.T, t = ft % g.T;
            if (warp == 0) {
                bool ok = true;
                if (lane == 0 && n >= 1) ok = mbar_wait_ab(bfull, (uint32_t)((n - 1) & 1), abort_flag);
                __syncwarp();
                if (*abort_flag || !ok) goto done;
                const float *om = omega + (size_t)ft * g.B * 2;
                float mx = 0.f;
                for (int e = lane; e < 2 * g.B; e += 32) {
                    const float v = om[e];
                    som[e] = v;
                    mx = fmaxf(mx, fabsf(v));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) {
                    float sc = 1.f;
                    if (ET == 1 && mx > 0.f && isfinite(mx)) {
                        int e;
                        frexpf(mx, &e);
                        sc = ldexpf(1.f, 14 - e);
                    }
                    *task_scale = sc;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(sready);
            }
            {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_ab(sready, (uint32_t)(n & 1), abort_flag);
                if (lane == 0 && ok && n >= 1) ok = mbar_wait_ab(bempty, (uint32_t)((n - 1) & 1), abort_flag);
                __syncwarp();
                if (*abort_flag || !ok) goto done;
            }
            const float sc = *task_scale;
            // B tile: row nrow = 2i (Re Y_i) or 2i+1 (Im Y_i); C_ij = omega_ij (i<j), conj(omega_ji) (i>j)
            for (int item = ptid; item < kused * nchunk; item += ADJ_PROD_WARPS * 32) {
                const int nrow = item / nchunk, kc = item % nchunk, i = nrow >> 1;
                const bool im_row = nrow & 1;
                float v[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jx = 4 * kc + q;
                    float cr = 0.f, ci = 0.f;
                    if (jx < g.A && jx != i) {
                        if (i < jx) { const int bb = pair_idx(i, jx, g.A); cr = som[2 * bb]; ci = som[2 * bb + 1]; }
                        else { const int bb = pair_idx(jx, i, g.A); cr = som[2 * bb]; ci = -som[2 * bb + 1]; }
                    }
                    cr *= sc;
                    ci *= sc;
                    v[2 * q] = im_row ? ci : cr;          // Re Y = Cr Er - Ci Ei ; Im Y = Ci Er + Cr Ei
                    v[2 * q + 1] = im_row ? cr : -ci;
                }
                uint4 hh, ll;
                Elem<ET>::split(v[0], v[1], hh.x, ll.x); Elem<ET>::split(v[2], v[3], hh.y, ll.y);
                Elem<ET>::split(v[4], v[5], hh.z, ll.z); Elem<ET>::split(v[6], v[7], hh.w, ll.w);
                const uint32_t off = (uint32_t)(kc >> 3) * b_atom + sw128_off(nrow, kc & 7);
                *reinterpret_cast<uint4 *>(bt_hi + off) = hh;
                if (X3) *reinterpret_cast<uint4 *>(bt_lo + off) = ll;
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bfull);
            // pixel chunks through the A-slot ring
            for (int c = 0; c < nchk; ++c, ++gs) {
                const int s = (int)(gs & 1);
                const long long use = gs >> 1;
                bool ok = true;
                if (lane == 0 && use >= 1) ok = mbar_wait_ab(empty0 + 8 * s, (uint32_t)((use - 1) & 1), abort_flag);
                __syncwarp();
                if (*abort_flag || !ok) goto done;
                uint8_t *ahi = gbase + (size_t)s * L.abuf_bytes, *alo = ahi + L.a_bytes;
                const int p0 = c * 128;
#pragma unroll 1
                for (int it = 0; it < nits; ++it) {
                    const int row = it_row[it], kc = it_kc[it], p = p0 + row;
                    const bool vp = p < g.npix;
                    float s6[6];
                    if (vp) load_s6(g, t, p, s6);
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int jx = 4 * kc + q;
                        float er = 0.f, ei = 0.f;
                        if (vp && jx < g.A) {
                            float k6[6];
#pragma unroll
                            for (int z = 0; z < 6; ++z) k6[z] = g.kap32[((size_t)f * g.A + jx) * 6 + z];
                            if (g.flat_array) phasor_of<!X3>(phase_frac<2>(k6, s6), er, ei);
                            else phasor_of<!X3>(phase_frac<3>(k6, s6), er, ei);
                        }
                        v[2 * q] = er;
                        v[2 * q + 1] = ei;
                    }
                    uint4 hh, ll;
                    Elem<ET>::split(v[0], v[1], hh.x, ll.x); Elem<ET>::split(v[2], v[3], hh.y, ll.y);
                    Elem<ET>::split(v[4], v[5], hh.z, ll.z); Elem<ET>::split(v[6], v[7], hh.w, ll.w);
                    const uint32_t off = (uint32_t)(kc >> 3) * a_atom + sw128_off(row, kc & 7);
                    *reinterpret_cast<uint4 *>(ahi + off) = hh;
                    if (X3) *reinterpret_cast<uint4 *>(alo + off) = ll;
                }
                if (ptid == 0) {
                    slot_scale[s] = sc;
                    slot_ft[s] = ft;
                    slot_p0[s] = p0;
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(full0 + 8 * s);
            }
        }
    } else if (warp == ADJ_MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, L.npad, Elem<ET>::kFmt);
            long long gs = 0, last = -1;
            int n = 0;
            for (int ft = blockIdx.x; ft < ntask; ft += gridDim.x, ++n) {
                if (!mbar_wait_ab(bfull, (uint32_t)(n & 1), abort_flag)) goto mma_done;
                for (int c = 0; c < nchk; ++c, ++gs) {
                    const int s = (int)(gs & 1);
                    if (!mbar_wait_ab(full0 + 8 * s, (uint32_t)((gs >> 1) & 1), abort_flag)) goto mma_done;
                    tc_fence_after();
                    const uint32_t sa_hi = base + (uint32_t)s * L.abuf_bytes, sa_lo = sa_hi + L.a_bytes;
                    const uint32_t sb_hi = base + L.b_off, sb_lo = sb_hi + L.b_bytes;
                    const uint32_t dcol = tmem0 + (uint32_t)(s * L.npad);
                    for (int kk = 0; kk < L.ksteps; ++kk) {
                        const uint32_t oa = (uint32_t)(kk >> 2) * a_atom + 32u * (kk & 3);
                        const uint32_t ob = (uint32_t)(kk >> 2) * b_atom + 32u * (kk & 3);
                        const uint64_t dah = sdesc_sw128(sa_hi + oa), dbh = sdesc_sw128(sb_hi + ob);
                        mma_bf16(dcol, dah, dbh, idesc, kk > 0 ? 1u : 0u);
                        if (X3) {
                            mma_bf16(dcol, dah, sdesc_sw128(sb_lo + ob), idesc, 1u);
                            mma_bf16(dcol, sdesc_sw128(sa_lo + oa), dbh, idesc, 1u);
                        }
                    }
                    mma_commit(dfull0 + 8 * s);
                    mma_commit(empty0 + 8 * s);
                    last = gs;
                }
                mma_commit(bempty);
            }
        mma_done:
            if (*abort_flag && last >= 0) {
                const int s = (int)(last & 1);
                long long t0 = clock64();
                while (clock64() - t0 < WAIT_CYCLES) {
                    uint32_t ok;
                    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                                 : "=r"(ok) : "r"(dfull0 + 8 * s), "r"((uint32_t)((last >> 1) & 1)) : "memory");
                    if (ok) break;
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 16-19)
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        long long gs = 0;
        for (int ft = blockIdx.x; ft < ntask; ft += gridDim.x) {
            for (int c = 0; c < nchk; ++c, ++gs) {
                const int s = (int)(gs & 1);
                const uint32_t par = (uint32_t)((gs >> 1) & 1);
                bool ok = true;
                if (lane == 0) ok = mbar_wait_ab(full0 + 8 * s, par, abort_flag);
                if (lane == 0 && ok) ok = mbar_wait_ab(dfull0 + 8 * s, par, abort_flag);
                __syncwarp();
                if (*abort_flag || !ok) goto done;
                tc_fence_after();
                const int ftm = slot_ft[s], p = slot_p0[s] + row;
                const float inv = 0.5f / slot_scale[s];
                const uint8_t *ahi = gbase + (size_t)s * L.abuf_bytes, *alo = ahi + L.a_bytes;
                float acc = 0.f;
                for (int c0 = 0; c0 < L.npad; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem0 + (uint32_t)(s * L.npad) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0, v);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kc = c0 / 8 + h;
                        if (kc >= nchunk) break;
                        const uint32_t off = (uint32_t)(kc >> 3) * a_atom + sw128_off(row, kc & 7);
                        const uint4 hv = *reinterpret_cast<const uint4 *>(ahi + off);
                        const uint4 lv = X3 ? *reinterpret_cast<const uint4 *>(alo + off) : make_uint4(0, 0, 0, 0);
                        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float2 eh = Elem<ET>::unpack(hw[q]), el = Elem<ET>::unpack(lw[q]);
                            acc += (eh.x + el.x) * v[8 * h + 2 * q] + (eh.y + el.y) * v[8 * h + 2 * q + 1];
                        }
                    }
                }
                if (p < g.npix) {
                    const int fe = ftm / g.T, te = ftm % g.T;
                    wbar[(size_t)ftm * g.npix + p] = pixel_w(g, fe, te, p) * inv * acc;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8 * s);
            }
        }
    }
done:
    __syncthreads();
    if (*abort_flag && tid == 0) atomicExch(g.status, (int)FM_ERR_TIMEOUT);
    if (warp == ADJ_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem0, (uint32_t)L.ncols);
    }
}

// xbar[f][p] = sum_t wbar[f][t][p] in a fixed order
__global__ void k_wbar_reduce(int F, int T, int npix, const float *__restrict__ wbar, float *__restrict__ xbar)
{
    const long long n = (long long)F * npix;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(e / npix), p = (int)(e % npix);
        const float *w = wbar + (size_t)f * T * npix + p;
        float s = 0.f;
        for (int t = 0; t < T; ++t) s += w[(size_t)t * npix];
        xbar[e] = s;
    }
}

static int g_num_sms = 0;

static int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

}  // namespace

template <int ET, bool X3>
static fm_status vis_tc_launch(Ctx &c, const FwdLayout &L, int rch, int sub, size_t smem, int grid, const float *x,
                               float *vis, cudaStream_t st)
{
    if (c.A <= 48) FM_CK(smem_opt_in(k_vis_tc<ET, X3, 3>));
    else FM_CK(smem_opt_in(k_vis_tc<ET, X3, 4>));
    return profiled(c, 0, st, [&]() -> fm_status {
        if (c.A <= 48) k_vis_tc<ET, X3, 3><<<grid, FWD_THREADS, smem, st>>>(c.g, L, rch, sub, x, c.tc_scale, vis);
        else k_vis_tc<ET, X3, 4><<<grid, FWD_THREADS, smem, st>>>(c.g, L, rch, sub, x, c.tc_scale, vis);
        FM_CK_LAUNCH();
        return FM_OK;
    });
}

fm_status launch_vis_tc(Ctx &c, const float *x, float *vis, cudaStream_t st)
{
    if (2 * c.A > 128) {
        set_error("the antenna-form tensor-core contraction supports at most 64 antennas");
        return FM_ERR_UNSUPPORTED;
    }
    const bool x3 = c.prec == FM_PREC_BF16X3 || c.prec == FM_PREC_FP16X3;
    const bool f16 = c.prec == FM_PREC_FP16X1 || c.prec == FM_PREC_FP16X3;
    FwdLayout L;
    L.npad = ((2 * c.A + 15) / 16) * 16;
    // channels per task (frequency recurrence), two TMEM accumulator sets of rch x npad
    // columns, enough tasks to fill the GPU
    int rch = 1;
    if (c.g.uniform_freq) {
        rch = 4;
        while (rch > 1 && (2 * rch * L.npad > 512 || (long long)c.T * ((c.F + rch - 1) / rch) < 4LL * num_sms())) --rch;
        if (const char *e = getenv("FM_TC_CHANNELS_PER_TASK")) {
            const int v = atoi(e);
            if (v >= 1) rch = v;
            while (rch > 1 && 2 * rch * L.npad > 512) --rch;
        }
        if (rch > c.F) rch = c.F;
    }
    L.ncols = 32;
    while (L.ncols < 2 * rch * L.npad) L.ncols *= 2;
    L.a_bytes = 128 * 128;
    L.b_bytes = (uint32_t)L.npad * 128;
    L.stage_bytes = (x3 ? 2u : 1u) * (L.a_bytes + L.b_bytes);
    const size_t vbytes = ((size_t)rch * c.B * 2 * 4 + 15) / 16 * 16;
    const size_t fixed = 1024 + vbytes + 16 * 4 + 64 + 64;
    const size_t budget = 226 * 1024;
    if (fixed >= budget) return FM_ERR_UNSUPPORTED;
    L.nstage = (int)((budget - fixed) / L.stage_bytes);
    if (L.nstage > 4) L.nstage = 4;
    if (L.nstage < 2) { set_error("forward tiles exceed shared memory"); return FM_ERR_UNSUPPORTED; }
    const size_t smem = 1024 + (size_t)L.nstage * L.stage_bytes + vbytes + 16 * L.nstage + 32 + 16;
    const int ntask = c.T * ((c.F + rch - 1) / rch);
    int grid = num_sms();
    if (grid > ntask) grid = ntask;
    // stages per TMEM accumulation chain (1024 pixels): bounds the accumulation error
    int sub = 16;
    if (const char *e = getenv("FM_TC_STAGES_PER_PARTIAL")) {
        const int v = atoi(e);
        if (v >= 1) sub = v;
    }
    if (f16) {
        k_chan_scale<<<c.F, 256, 0, st>>>(c.npix, x, c.domega_max, c.tc_scale);
        FM_CK_LAUNCH();
        return x3 ? vis_tc_launch<1, true>(c, L, rch, sub, smem, grid, x, vis, st)
                  : vis_tc_launch<1, false>(c, L, rch, sub, smem, grid, x, vis, st);
    }
    return x3 ? vis_tc_launch<0, true>(c, L, rch, sub, smem, grid, x, vis, st)
              : vis_tc_launch<0, false>(c, L, rch, sub, smem, grid, x, vis, st);
}

template <int ET, bool X3>
static fm_status adj_tc_launch(Ctx &c, const AdjLayout &L, size_t smem, int grid, const float *omega, float *wbar,
                               cudaStream_t st)
{
    FM_CK(smem_opt_in(k_adj_tc<ET, X3>));
    return profiled(c, 1, st, [&]() -> fm_status {
        k_adj_tc<ET, X3><<<grid, ADJ_THREADS, smem, st>>>(c.g, L, omega, wbar);
        FM_CK_LAUNCH();
        return FM_OK;
    });
}

fm_status launch_adjoint_tc(Ctx &c, const float *omega, float *xbar, cudaStream_t st)
{
    if (2 * c.A > 128) {
        set_error("the antenna-form tensor-core adjoint supports at most 64 antennas");
        return FM_ERR_UNSUPPORTED;
    }
    if (!c.tc_wbar) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(float) * (size_t)c.F * c.T * c.npix) != cudaSuccess) {
            set_error("cudaMalloc of the adjoint pixel-weight buffer failed");
            return FM_ERR_ALLOC;
        }
        c.allocs.push_back(p);
        c.tc_wbar = (float *)p;
    }
    const bool x3 = c.prec == FM_PREC_BF16X3 || c.prec == FM_PREC_FP16X3;
    const bool f16 = c.prec == FM_PREC_FP16X1 || c.prec == FM_PREC_FP16X3;
    AdjLayout L;
    L.npad = ((2 * c.A + 15) / 16) * 16;
    L.ksteps = (2 * c.A + 15) / 16;
    L.katoms = (L.ksteps + 3) / 4;
    L.ncols = 32;
    while (L.ncols < ADJ_SLOTS * L.npad) L.ncols *= 2;
    L.a_bytes = (uint32_t)L.katoms * 128u * 128u;
    L.b_bytes = (uint32_t)L.katoms * (uint32_t)L.npad * 128u;
    L.abuf_bytes = (x3 ? 2u : 1u) * L.a_bytes;
    L.b_off = ADJ_SLOTS * L.abuf_bytes;
    L.om_off = L.b_off + (x3 ? 2u : 1u) * L.b_bytes;
    L.meta_off = L.om_off + (uint32_t)((2 * sizeof(float) * (size_t)c.B + 15) / 16 * 16);
    const size_t smem = 1024 + (size_t)L.meta_off + 64 + 72 + 16;
    if (smem > 227 * 1024) { set_error("adjoint tiles exceed shared memory"); return FM_ERR_UNSUPPORTED; }
    const int ntask = c.F * c.T;
    int grid = num_sms();
    if (grid > ntask) grid = ntask;
    fm_status s;
    if (f16)
        s = x3 ? adj_tc_launch<1, true>(c, L, smem, grid, omega, c.tc_wbar, st)
               : adj_tc_launch<1, false>(c, L, smem, grid, omega, c.tc_wbar, st);
    else
        s = x3 ? adj_tc_launch<0, true>(c, L, smem, grid, omega, c.tc_wbar, st)
               : adj_tc_launch<0, false>(c, L, smem, grid, omega, c.tc_wbar, st);
    if (s != FM_OK) return s;
    k_wbar_reduce<<<1024, 256, 0, st>>>(c.F, c.T, c.npix, c.tc_wbar, xbar);
    FM_CK_LAUNCH();
    return FM_OK;
}

}  // namespace fm
