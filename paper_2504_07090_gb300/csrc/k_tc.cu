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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int TC_THREADS = 256;
constexpr int KST = 64;                               // pixels per stage (one swizzle row of bf16)
constexpr long long WAIT_CYCLES = 4000000000LL;       // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > WAIT_CYCLES) return false;
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)1u << 16;                           // leading offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                 // stride between 8-row groups
    d |= (uint64_t)1u << 46;                           // descriptor version for tcgen05
    d |= (uint64_t)2u << 61;                           // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of the 16-byte chunk `chunk` (0..7) of row `row` in a 128B-swizzled tile.
__device__ __forceinline__ uint32_t sw128_off(int row, int chunk)
{
    return (uint32_t)row * 128u + ((uint32_t)(chunk ^ (row & 7)) << 4);
}

__device__ __forceinline__ uint32_t u32_of(const void *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Operand element type: 0 = BF16 (unscaled), 1 = FP16 (power-of-two scaled operands).
template <int ET> struct Elem;
template <> struct Elem<0> {
    static constexpr uint32_t kFmt = 1;   // instruction-descriptor format code of BF16
    static __device__ __forceinline__ void split(float a, float b, uint32_t &hi, uint32_t &lo)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        float2 hf = __bfloat1622float2(h);
        __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = u32_of(&h);
        lo = u32_of(&l);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t w)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
    }
};
template <> struct Elem<1> {
    static constexpr uint32_t kFmt = 0;   // FP16
    static __device__ __forceinline__ void split(float a, float b, uint32_t &hi, uint32_t &lo)
    {
        __half2 h = __floats2half2_rn(a, b);
        float2 hf = __half22float2(h);
        __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = u32_of(&h);
        lo = u32_of(&l);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t w)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
};

// Instruction descriptor, kind::f16: FP32 accumulator, A and B of format `fmt`, K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float phase_frac(const float *kap, const float *s)
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

// E = exp(-2 pi i frac)
__device__ __forceinline__ void phasor_of(float fr, float &er, float &ei)
{
    float sn, cs;
    sincos_turns(fr, sn, cs);
    er = cs;
    ei = -sn;
}

__device__ __forceinline__ float pixel_w(const DevGeom &g, int f, int t, int p)
{
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
template <int ET, bool X3, int KMAX>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_vis_tc(DevGeom g, FwdLayout L, int rch, const float *__restrict__ x, const float *__restrict__ chan_scale,
         float *__restrict__ vis)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;                 // 1024-aligned for the swizzle atoms
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + L.nstage * L.stage_bytes;        // nstage mbarriers (8 B each)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + L.nstage * L.stage_bytes + 8 * L.nstage);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows_used = 2 * g.A;
    const int ntl = X3 ? 2 : 1;

    for (int s = 0; s < L.nstage; ++s) {            // zero the padding rows once
        uint8_t *st = gbase + (size_t)s * L.stage_bytes;
        for (int tl = 0; tl < ntl; ++tl) {
            uint8_t *ta = st + tl * L.a_bytes;
            for (int e = tid; e < (128 - rows_used) * 8; e += TC_THREADS)
                reinterpret_cast<uint4 *>(ta + (size_t)(rows_used + e / 8) * 128)[e % 8] = make_uint4(0, 0, 0, 0);
            uint8_t *tb = st + ntl * L.a_bytes + tl * L.b_bytes;
            for (int e = tid; e < (L.npad - rows_used) * 8; e += TC_THREADS)
                reinterpret_cast<uint4 *>(tb + (size_t)(rows_used + e / 8) * 128)[e % 8] = make_uint4(0, 0, 0, 0);
        }
    }
    if (tid == 0) {
        for (int s = 0; s < L.nstage; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(su32(tmem_slot), (uint32_t)L.ncols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;
    const uint32_t idesc = idesc_f16(128, L.npad, Elem<ET>::kFmt);
    const uint32_t wsub = (uint32_t)(lane & 3) * 4u;               // byte offset of this lane's word in a chunk
    const int wchunk = lane >> 2;                                   // 16-byte chunk holding pixels 2l, 2l+1

    const int nst = (g.npix + KST - 1) / KST;
    const int ngrp = (g.F + rch - 1) / rch;
    const int ntask = ngrp * g.T;
    long long gs = 0;
    int last_s = -1;
    long long last_use = 0;
    bool aborted = false;

    for (int task = blockIdx.x; task < ntask && !aborted; task += gridDim.x) {
        const int t = task % g.T, f0 = (task / g.T) * rch;
        const int nr = min(rch, g.F - f0);
        for (int j = 0; j < nst && !aborted; ++j) {
            const int pa = j * KST + 2 * lane, pb = pa + 1;
            const bool va = pa < g.npix, vb = pb < g.npix;
            float sa[6], sb[6];
            if (va) load_s6(g, t, pa, sa);
            if (vb) load_s6(g, t, pb, sb);
            // phasor state of this thread's antennas at its two pixels, advanced by D per channel
            float er[KMAX][2], ei[KMAX][2], dr[KMAX][2], di[KMAX][2];
            for (int r = 0; r < nr; ++r, ++gs) {
                const int f = f0 + r;
                const int s = (int)(gs % L.nstage);
                const long long use = gs / L.nstage;
                const float scale = ET == 1 ? chan_scale[f] : 1.f;
                const float wa = va ? pixel_w(g, f, t, pa) * x[(size_t)f * g.npix + pa] * scale : 0.f;
                const float wb = vb ? pixel_w(g, f, t, pb) * x[(size_t)f * g.npix + pb] * scale : 0.f;
#pragma unroll
                for (int k = 0; k < KMAX; ++k) {
                    const int i = warp + 8 * k;
                    if (i >= g.A) continue;
                    if (r == 0) {
                        float k6[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) k6[q] = g.kap32[((size_t)f * g.A + i) * 6 + q];
                        er[k][0] = ei[k][0] = er[k][1] = ei[k][1] = 0.f;
                        if (va) phasor_of(phase_frac(k6, sa), er[k][0], ei[k][0]);
                        if (vb) phasor_of(phase_frac(k6, sb), er[k][1], ei[k][1]);
                        if (nr > 1) {
                            const float d0 = g.dkap32[3 * i], d1 = g.dkap32[3 * i + 1], d2 = g.dkap32[3 * i + 2];
                            phasor_of(d0 * (sa[0] + sa[1]) + d1 * (sa[2] + sa[3]) + d2 * (sa[4] + sa[5]), dr[k][0], di[k][0]);
                            phasor_of(d0 * (sb[0] + sb[1]) + d1 * (sb[2] + sb[3]) + d2 * (sb[4] + sb[5]), dr[k][1], di[k][1]);
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
                bool bad = false;
                if (tid == 0 && use >= 1) bad = !mbar_wait(bar0 + 8 * s, (uint32_t)((use - 1) & 1));
                if (__syncthreads_or(bad)) { aborted = true; break; }
                uint8_t *st = gbase + (size_t)s * L.stage_bytes;
                uint8_t *a_hi = st, *a_lo = st + L.a_bytes;
                uint8_t *b_hi = st + ntl * L.a_bytes, *b_lo = b_hi + L.b_bytes;
#pragma unroll
                for (int k = 0; k < KMAX; ++k) {
                    const int i = warp + 8 * k;
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
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t sa_hi = base + (uint32_t)s * L.stage_bytes;
                    const uint32_t sa_lo = sa_hi + L.a_bytes;
                    const uint32_t sb_hi = sa_hi + (uint32_t)ntl * L.a_bytes;
                    const uint32_t sb_lo = sb_hi + L.b_bytes;
                    const uint32_t dacc = tmem_d + (uint32_t)(r * L.npad);
#pragma unroll
                    for (int kk = 0; kk < KST / 16; ++kk) {
                        const uint32_t off = 32u * kk;
                        const uint64_t dah = sdesc_sw128(sa_hi + off), dbh = sdesc_sw128(sb_hi + off);
                        mma_bf16(dacc, dah, dbh, idesc, (j > 0 || kk > 0) ? 1u : 0u);
                        if (X3) {
                            mma_bf16(dacc, dah, sdesc_sw128(sb_lo + off), idesc, 1u);
                            mma_bf16(dacc, sdesc_sw128(sa_lo + off), dbh, idesc, 1u);
                        }
                    }
                    mma_commit(bar0 + 8 * s);
                }
                last_s = s;
                last_use = use;
            }
        }
        if (aborted) break;
        bool bad = false;
        if (tid == 0) bad = !mbar_wait(bar0 + 8 * last_s, (uint32_t)(last_use & 1));
        if (__syncthreads_or(bad)) { aborted = true; break; }
        if (warp < 4) {
            tc_fence_after();
            const int row = 32 * warp + lane;
            const int i = row >> 1;
            const bool even = (row & 1) == 0;
            for (int r = 0; r < nr; ++r) {
                const int f = f0 + r;
                const float inv = ET == 1 ? 1.f / chan_scale[f] : 1.f;
                const size_t ft = (size_t)f * g.T + t;
                for (int c0 = 0; c0 < L.npad; c0 += 16) {
                    float v[16], pv[16];
                    tmem_ld16(tmem_d + ((uint32_t)(32 * warp) << 16) + (uint32_t)(r * L.npad + c0), v);
#pragma unroll
                    for (int q = 0; q < 16; ++q) pv[q] = __shfl_xor_sync(0xffffffffu, v[q], 1);
                    if (even && i < g.A) {
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int jn = c0 / 2 + jj;
                            if (jn > i && jn < g.A) {
                                const size_t o = (ft * g.B + pair_idx(i, jn, g.A)) * 2;
                                vis[o] = (v[2 * jj] + pv[2 * jj + 1]) * inv;
                                vis[o + 1] = (pv[2 * jj] - v[2 * jj + 1]) * inv;
                            }
                        }
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (aborted) {
        if (tid == 0) {
            atomicExch(g.status, (int)FM_ERR_TIMEOUT);
            if (last_s >= 0) mbar_wait(bar0 + 8 * last_s, (uint32_t)(last_use & 1));   // drain own MMAs (bounded)
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_d, (uint32_t)L.ncols);
    }
}

// ------------------------------------------------------------------ adjoint kernel
struct AdjLayout {
    int npad, katoms, ksteps, ncols;
    uint32_t a_bytes, b_bytes, buf_bytes;     // per hi (or lo) tile; buffer = [A_hi A_lo B_hi B_lo]
};

template <int ET, bool X3>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_adj_tc(DevGeom g, AdjLayout L, const float *__restrict__ omega, float *__restrict__ xbar)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + 2 * L.buf_bytes;                 // 2 mbarriers
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + 2 * L.buf_bytes + 16);
    float *sscale = reinterpret_cast<float *>(gbase + 2 * L.buf_bytes + 32);   // [2] B-operand scale per buffer
    float *sred = sscale + 2;                                                     // [8] warp maxima
    float *som = reinterpret_cast<float *>(gbase + 2 * L.buf_bytes + 128);       // [2B] omega of this (f, t)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kused = 2 * g.A;
    const int ntl = X3 ? 2 : 1;
    const uint32_t a_atom = 128u * 128u, b_atom = (uint32_t)L.npad * 128u;

    for (uint32_t e = tid; e < 2 * L.buf_bytes / 16; e += TC_THREADS)
        reinterpret_cast<uint4 *>(gbase)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(su32(tmem_slot), (uint32_t)L.ncols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem0 = *tmem_slot;
    const uint32_t idesc = idesc_f16(128, L.npad, Elem<ET>::kFmt);
    const int ntile = (g.npix + 127) / 128;
    const int ntask = g.F * ntile;
    const int nchunk = (kused + 7) / 8;            // 16-byte chunks of K actually used
    const int half = (nchunk + 1) / 2;             // A-tile chunks per thread (two threads per pixel row)
    long long gi = 0;
    bool aborted = false;
    long long pending = -1;
    long long last_issued = -1;

    auto epilogue = [&](long long it, int f, int t, int p0, float &xacc) -> bool {
        const int b = (int)(it & 1);
        bool bad = false;
        if (tid == 0) bad = !mbar_wait(bar0 + 8 * b, (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(bad)) return false;
        if (warp < 4) {
            tc_fence_after();
            const int row = 32 * warp + lane, p = p0 + row;
            const uint8_t *ahi = gbase + (size_t)b * L.buf_bytes, *alo = ahi + L.a_bytes;
            float acc = 0.f;
            for (int c0 = 0; c0 < L.npad; c0 += 16) {
                float v[16];
                tmem_ld16(tmem0 + (uint32_t)(b * L.npad) + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
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
            if (p < g.npix) xacc += pixel_w(g, f, t, p) * (0.5f / sscale[b]) * acc;
        }
        tc_fence_before();
        __syncthreads();
        return true;
    };

    for (int task = blockIdx.x; task < ntask && !aborted; task += gridDim.x) {
        const int f = task / ntile, p0 = (task % ntile) * 128;
        float xacc = 0.f;
        for (int t = 0; t < g.T; ++t, ++gi) {
            const int b = (int)(gi & 1);
            // omega of (f, t) into shared memory and its largest component
            const float *om = omega + (size_t)(f * g.T + t) * g.B * 2;
            float mx = 0.f;
            for (int e = tid; e < 2 * g.B; e += TC_THREADS) {
                const float v = om[e];
                som[e] = v;
                mx = fmaxf(mx, fabsf(v));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) sred[warp] = mx;
            __syncthreads();
            if (tid == 0) {
                float m = 0.f;
                for (int w = 0; w < TC_THREADS / 32; ++w) m = fmaxf(m, sred[w]);
                float sc = 1.f;
                if (ET == 1 && m > 0.f && isfinite(m)) {
                    int e;
                    frexpf(m, &e);
                    sc = ldexpf(1.f, 14 - e);
                }
                sscale[b] = sc;
            }
            uint8_t *ahi = gbase + (size_t)b * L.buf_bytes, *alo = ahi + L.a_bytes;
            uint8_t *bhi = ahi + ntl * L.a_bytes, *blo = bhi + L.b_bytes;
            {   // A tile: row = pixel, chunk kc = (Re E_j, Im E_j) for j = 4kc .. 4kc+3
                const int row = tid & 127, hsel = tid >> 7, p = p0 + row;
                float s6[6];
                const bool vp = p < g.npix;
                if (vp) load_s6(g, t, p, s6);
                const int kc0 = hsel * half, kc1 = min(nchunk, kc0 + half);
                for (int kc = kc0; kc < kc1; ++kc) {
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int jx = 4 * kc + q;
                        float er = 0.f, ei = 0.f;
                        if (vp && jx < g.A) {
                            float k6[6];
#pragma unroll
                            for (int z = 0; z < 6; ++z) k6[z] = g.kap32[((size_t)f * g.A + jx) * 6 + z];
                            phasor_of(phase_frac(k6, s6), er, ei);
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
            }
            __syncthreads();   // som and sscale visible
            {   // B tile: row n = 2i (Re Y_i) or 2i+1 (Im Y_i); C_ij = omega_ij (i<j), conj(omega_ji) (i>j)
                const float sc = sscale[b];
                for (int item = tid; item < kused * nchunk; item += TC_THREADS) {
                    const int n = item / nchunk, kc = item % nchunk, i = n >> 1;
                    const bool im_row = n & 1;
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
                    const uint32_t off = (uint32_t)(kc >> 3) * b_atom + sw128_off(n, kc & 7);
                    *reinterpret_cast<uint4 *>(bhi + off) = hh;
                    if (X3) *reinterpret_cast<uint4 *>(blo + off) = ll;
                }
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t sa_hi = base + (uint32_t)b * L.buf_bytes, sa_lo = sa_hi + L.a_bytes;
                const uint32_t sb_hi = sa_hi + (uint32_t)ntl * L.a_bytes, sb_lo = sb_hi + L.b_bytes;
                const uint32_t dcol = tmem0 + (uint32_t)(b * L.npad);
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
                mma_commit(bar0 + 8 * b);
            }
            last_issued = gi;
            if (pending >= 0) {
                if (!epilogue(pending, f, t - 1, p0, xacc)) { aborted = true; break; }
            }
            pending = gi;
        }
        if (aborted) break;
        if (!epilogue(pending, f, g.T - 1, p0, xacc)) { aborted = true; break; }
        pending = -1;
        if (warp < 4) {
            const int p = p0 + 32 * warp + lane;
            if (p < g.npix) xbar[(size_t)f * g.npix + p] = xacc;
        }
    }
    if (aborted) {
        if (tid == 0) {
            atomicExch(g.status, (int)FM_ERR_TIMEOUT);
            if (last_issued >= 0) mbar_wait(bar0 + 8 * (last_issued & 1), (uint32_t)((last_issued >> 1) & 1));
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem0, (uint32_t)L.ncols);
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
static fm_status vis_tc_launch(Ctx &c, const FwdLayout &L, int rch, size_t smem, int grid, const float *x, float *vis,
                               cudaStream_t st)
{
    if (c.A <= 40) {
        FM_CK(cudaFuncSetAttribute(k_vis_tc<ET, X3, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vis_tc<ET, X3, 5><<<grid, TC_THREADS, smem, st>>>(c.g, L, rch, x, c.tc_scale, vis);
    } else {
        FM_CK(cudaFuncSetAttribute(k_vis_tc<ET, X3, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vis_tc<ET, X3, 8><<<grid, TC_THREADS, smem, st>>>(c.g, L, rch, x, c.tc_scale, vis);
    }
    FM_CK_LAUNCH();
    return FM_OK;
}

fm_status launch_vis_tc(Ctx &c, const float *x, float *vis, cudaStream_t st)
{
    if (2 * c.A > 128) {
        set_error("tensor-core contraction supports at most 64 antennas in this build");
        return FM_ERR_UNSUPPORTED;
    }
    const bool x3 = c.prec == FM_PREC_BF16X3 || c.prec == FM_PREC_FP16X3;
    const bool f16 = c.prec == FM_PREC_FP16X1 || c.prec == FM_PREC_FP16X3;
    FwdLayout L;
    L.npad = ((2 * c.A + 15) / 16) * 16;
    // channels per task (frequency recurrence): enough tasks to fill the GPU, TMEM for rch accumulators
    int rch = 1;
    if (c.g.uniform_freq) {
        rch = 4;
        while (rch > 1 && (rch * L.npad > 512 || (long long)c.T * ((c.F + rch - 1) / rch) < 4LL * num_sms())) --rch;
        if (rch > c.F) rch = c.F;
    }
    L.ncols = 32;
    while (L.ncols < rch * L.npad) L.ncols *= 2;
    L.a_bytes = 128 * 128;
    L.b_bytes = (uint32_t)L.npad * 128;
    L.stage_bytes = (x3 ? 2u : 1u) * (L.a_bytes + L.b_bytes);
    const size_t budget = 225 * 1024;
    L.nstage = (int)((budget - 1024 - 64) / L.stage_bytes);
    if (L.nstage > 4) L.nstage = 4;
    if (L.nstage < 2) return FM_ERR_UNSUPPORTED;
    const size_t smem = 1024 + (size_t)L.nstage * L.stage_bytes + 8 * L.nstage + 16;
    const int ntask = c.T * ((c.F + rch - 1) / rch);
    int grid = num_sms();
    if (grid > ntask) grid = ntask;
    if (f16) {
        k_chan_scale<<<c.F, 256, 0, st>>>(c.npix, x, c.domega_max, c.tc_scale);
        FM_CK_LAUNCH();
        return x3 ? vis_tc_launch<1, true>(c, L, rch, smem, grid, x, vis, st)
                  : vis_tc_launch<1, false>(c, L, rch, smem, grid, x, vis, st);
    }
    return x3 ? vis_tc_launch<0, true>(c, L, rch, smem, grid, x, vis, st)
              : vis_tc_launch<0, false>(c, L, rch, smem, grid, x, vis, st);
}

template <int ET, bool X3>
static fm_status adj_tc_launch(Ctx &c, const AdjLayout &L, size_t smem, int grid, const float *omega, float *xbar,
                               cudaStream_t st)
{
    FM_CK(cudaFuncSetAttribute(k_adj_tc<ET, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_adj_tc<ET, X3><<<grid, TC_THREADS, smem, st>>>(c.g, L, omega, xbar);
    FM_CK_LAUNCH();
    return FM_OK;
}

fm_status launch_adjoint_tc(Ctx &c, const float *omega, float *xbar, cudaStream_t st)
{
    if (2 * c.A > 128) {
        set_error("tensor-core adjoint supports at most 64 antennas in this build");
        return FM_ERR_UNSUPPORTED;
    }
    const bool x3 = c.prec == FM_PREC_BF16X3 || c.prec == FM_PREC_FP16X3;
    const bool f16 = c.prec == FM_PREC_FP16X1 || c.prec == FM_PREC_FP16X3;
    AdjLayout L;
    L.npad = ((2 * c.A + 15) / 16) * 16;
    L.ksteps = (2 * c.A + 15) / 16;
    L.katoms = (L.ksteps + 3) / 4;
    L.ncols = 32;
    while (L.ncols < 2 * L.npad) L.ncols *= 2;
    L.a_bytes = (uint32_t)L.katoms * 128u * 128u;
    L.b_bytes = (uint32_t)L.katoms * (uint32_t)L.npad * 128u;
    L.buf_bytes = (x3 ? 2u : 1u) * (L.a_bytes + L.b_bytes);
    const size_t smem = 1024 + 2 * (size_t)L.buf_bytes + 128 + 2 * sizeof(float) * (size_t)c.B;
    if (smem > 227 * 1024) { set_error("adjoint tiles exceed shared memory"); return FM_ERR_UNSUPPORTED; }
    const int ntask = c.F * ((c.npix + 127) / 128);
    int grid = num_sms();
    if (grid > ntask) grid = ntask;
    if (f16)
        return x3 ? adj_tc_launch<1, true>(c, L, smem, grid, omega, xbar, st) : adj_tc_launch<1, false>(c, L, smem, grid, omega, xbar, st);
    return x3 ? adj_tc_launch<0, true>(c, L, smem, grid, omega, xbar, st) : adj_tc_launch<0, false>(c, L, smem, grid, omega, xbar, st);
}

}  // namespace fm
