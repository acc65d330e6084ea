// Mode <-> pixel transforms on the tensor cores (sm_103a tcgen05), Eq. (fg_separable):
//   forward  x[f][d][r] = sum_m Phi[r][m] W[d][m],   W[d][m] = sum_n Leg[d][n] a[f][m][n]
//   adjoint  abar[f][m][n] = sum_d U[m][d] Leg[d][n],  U[m][d] = sum_r Phi[r][m] xbar[f][d][r]
// Each direction is two chained GEMMs in one CTA per (channel, 128-row tile): the first
// product accumulates in TMEM, is scaled by a power of two, split into FP16 hi/lo parts
// and written to shared memory as the A operand of the second product.  Every operand is
// used in its natural K-major layout (no transposes at run time): the basis tables and
// their transposes are prepared once per handle as 128-byte-swizzled FP16 hi/lo images,
// the modes a and the pixel gradient xbar are converted tile by tile.  Products use the
// three-term split hi*hi + hi*lo + lo*hi with FP32 accumulation.
//
// K is processed one 64-wide atom at a time through one or two operand slots: the image
// atom arrives by bulk copy, the other operand is converted by all threads, and one thread
// issues 4 x 3 MMAs per atom and commits them to the slot's mbarrier; a slot is refilled
// once the barrier shows its MMAs complete (bounded waits throughout).
#include <cmath>
#include <cstdlib>

#include "fm_internal.cuh"
#include "tc_ptx.cuh"

namespace fm {
namespace {

using namespace tc;

constexpr int MD_THREADS = 256;
constexpr float MD_CSCALE = 16384.f;     // basis tables (|value| <= 1) are stored times 2^14

struct MdDims {
    int F, M, N, R, D;         // modes (RA, Dec), pixels (RA, Dec)
    int Mp, Np, Rp, Dp;        // padded to multiples of 64
};

// 128-byte-swizzled K-major atom: element (row, k) of a [rows][64] atom at byte offset
__device__ __forceinline__ uint32_t atom_off(int row, int k)
{
    return (uint32_t)row * 128u + ((uint32_t)(((k >> 3) ^ (row & 7))) << 4) + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void split_h(float v, __half &h, __half &l)
{
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
}

// image of an operand [rows_pad][k_pad]: per 64-wide K atom, the hi rows then the lo rows
// (element (row, k) = scale * (transpose ? src[k][row0 + row] : src[row0 + row][k]), zero
// outside the source)
__global__ void k_md_image(const double *__restrict__ src, int src_rows, int src_cols, int transpose, int row0,
                           int rows_pad, int k_pad, float scale, uint8_t *__restrict__ img)
{
    const long long total = (long long)rows_pad * k_pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e / k_pad), k = (int)(e % k_pad);
        const int sr = transpose ? k : row0 + row, sc = transpose ? row0 + row : k;
        const double v = (sr < src_rows && sc < src_cols) ? src[(size_t)sr * src_cols + sc] : 0.0;
        __half h, l;
        split_h((float)(v * scale), h, l);
        uint8_t *atom = img + (size_t)(k >> 6) * 2 * rows_pad * 128;
        *reinterpret_cast<__half *>(atom + atom_off(row, k & 63)) = h;
        *reinterpret_cast<__half *>(atom + (size_t)rows_pad * 128 + atom_off(row, k & 63)) = l;
    }
}

__device__ __forceinline__ float block_max(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    float m = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
    return m;
}

__device__ __forceinline__ float pow2_below(float mx)
{
    float sc = 1.f;
    if (mx > 0.f && isfinite(mx)) {
        int e;
        frexpf(mx, &e);
        sc = ldexpf(1.f, 14 - e);
    }
    return sc;
}

// One K atom: A (128 rows) and B (nrows rows) tiles are in shared memory at a_s / b_s,
// hi rows then lo rows; D[tmem] (+)= A B^T over the atom's 64 K values.
__device__ __forceinline__ void issue_atom(uint32_t tmem, uint32_t a_s, uint32_t b_s, int nrows, bool first,
                                           uint32_t idesc)
{
    const uint32_t a_lo = a_s + 128u * 128u, b_lo = b_s + (uint32_t)nrows * 128u;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint64_t dah = sdesc_sw128(a_s + 32u * kk), dbh = sdesc_sw128(b_s + 32u * kk);
        mma_bf16(tmem, dah, dbh, idesc, (first && kk == 0) ? 0u : 1u);
        mma_bf16(tmem, dah, sdesc_sw128(b_lo + 32u * kk), idesc, 1u);
        mma_bf16(tmem, sdesc_sw128(a_lo + 32u * kk), dbh, idesc, 1u);
    }
}

// Shared state of both kernels: one or two operand slots, each an A atom (128 rows) and a B
// atom (up to b_rows_max rows), hi rows then lo rows; per slot one mbarrier for the bulk copy
// of its basis-image atom and one for the MMAs that read it.
struct MdSmem {
    uint8_t *g;                // slot 0's A atom; its B atom follows at +32 KB
    uint32_t base;             // its shared address
    uint32_t stride;           // bytes from slot 0 to slot 1 (0 with one slot)
    uint32_t bars;             // bar_img(s) = bars + 8 s, bar_mma(s) = bars + 16 + 8 s
    uint32_t *tmem_slot;
    volatile int *abort_flag;
    float *red;
    __device__ __forceinline__ uint8_t *a(int s) const { return g + (uint32_t)s * stride; }
    __device__ __forceinline__ uint8_t *b(int s) const { return g + (uint32_t)s * stride + 2 * 128 * 128; }
    __device__ __forceinline__ uint32_t a_s(int s) const { return base + (uint32_t)s * stride; }
    __device__ __forceinline__ uint32_t b_s(int s) const { return base + (uint32_t)s * stride + 2u * 128u * 128u; }
    __device__ __forceinline__ uint32_t bar_img(int s) const { return bars + 8u * (uint32_t)s; }
    __device__ __forceinline__ uint32_t bar_mma(int s) const { return bars + 16u + 8u * (uint32_t)s; }
};

__host__ __device__ constexpr uint32_t md_slot_bytes(int b_rows_max)
{
    return 2u * 128u * 128u + 2u * (uint32_t)b_rows_max * 128u;
}

__device__ __forceinline__ MdSmem md_smem(int b_rows_max, int ns)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t slot = md_slot_bytes(b_rows_max), tail = (uint32_t)ns * slot;
    MdSmem m;
    m.g = smem_raw + (base - raw);
    m.base = base;
    m.stride = ns == 2 ? slot : 0u;
    m.bars = base + tail;
    m.tmem_slot = reinterpret_cast<uint32_t *>(m.g + tail + 32);
    m.abort_flag = reinterpret_cast<volatile int *>(m.g + tail + 36);
    m.red = reinterpret_cast<float *>(m.g + tail + 64);
    return m;
}

// after an atom is filled: make the generic-proxy writes visible to the tensor core
__device__ __forceinline__ void md_filled()
{
    fence_async_smem();
    __syncthreads();
}

// largest |v| over a row-major [rows][cols] array (16-byte loads when rows are 16-byte
// aligned, eight in flight per thread); every thread receives the result
__device__ __forceinline__ float md_absmax(const float *a, int rows, int cols, bool skip_first, float *red)
{
    float m = 0.f;
    const long long n = (long long)rows * cols;
    if ((cols & 3) == 0) {
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        const long long n4 = n / 4;
        for (long long e0 = threadIdx.x; e0 < n4; e0 += 8LL * blockDim.x) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const long long e = e0 + (long long)u * blockDim.x;
                v[u] = e < n4 ? __ldg(a4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const long long e = e0 + (long long)u * blockDim.x;
                const float x0 = (skip_first && e == 0) ? 0.f : v[u].x;
                m = fmaxf(m, fmaxf(fmaxf(fabsf(x0), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
            }
        }
    } else {
        for (long long e = threadIdx.x; e < n; e += blockDim.x)
            if (!(skip_first && e == 0)) m = fmaxf(m, fabsf(__ldg(a + e)));
    }
    return block_max(m, red);
}

// B operand atom from a row-major FP32 matrix src [rows][cols] (rows_pad rows, K values
// 64 ka .. 64 ka + 63), scaled and split into FP16 hi / lo rows; entry (0, 0) is read as
// zero when zero00.  16-byte loads (eight in flight) when cols is a multiple of 4.
__device__ __forceinline__ void md_convert_atom(const float *src, int rows, int cols, int rows_pad, int ka,
                                                float sc, bool zero00, uint8_t *b)
{
    const int n4 = rows_pad * 16;                  // 4-value pieces in the atom
    const bool vec = (cols & 3) == 0;
    for (int e0 = threadIdx.x; e0 < n4; e0 += 8 * blockDim.x) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            const int row = e >> 4, k = 64 * ka + 4 * (e & 15);
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < n4 && row < rows) {
                const float *p = src + (size_t)row * cols + k;
                if (vec && k + 3 < cols) x = __ldg(reinterpret_cast<const float4 *>(p));
                else {
                    if (k < cols) x.x = __ldg(p);
                    if (k + 1 < cols) x.y = __ldg(p + 1);
                    if (k + 2 < cols) x.z = __ldg(p + 2);
                    if (k + 3 < cols) x.w = __ldg(p + 3);
                }
                if (zero00 && row == 0 && k == 0) x.x = 0.f;
            }
            v[u] = x;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= n4) break;
            const int row = e >> 4, k = 4 * (e & 15);
            __half h0, l0, h1, l1, h2, l2, h3, l3;
            split_h(v[u].x * sc, h0, l0);
            split_h(v[u].y * sc, h1, l1);
            split_h(v[u].z * sc, h2, l2);
            split_h(v[u].w * sc, h3, l3);
            const uint32_t off = atom_off(row, k);     // 4 consecutive K values stay in one 16-byte chunk
            auto pk = [](__half lo16, __half hi16) {
                return (uint32_t)__half_as_ushort(lo16) | ((uint32_t)__half_as_ushort(hi16) << 16);
            };
            *reinterpret_cast<uint2 *>(b + off) = make_uint2(pk(h0, h1), pk(h2, h3));
            *reinterpret_cast<uint2 *>(b + (size_t)rows_pad * 128 + off) = make_uint2(pk(l0, l1), pk(l2, l3));
        }
    }
}

// TMEM accumulator (128 lanes x ncols columns at column c0) -> scaled FP16 hi/lo A atom
// for K atom ka of the next product; warps w and w + 4 share lane quarter w & 3 and take
// alternate 16-column groups
__device__ __forceinline__ void md_tmem_to_atom(uint32_t tmem, int c0, int ka, float sc, uint8_t *a)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = w & 3, half = w >> 2;
    const int row = 32 * quarter + lane;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(c0 + 64 * ka);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int cg = 16 * (2 * g + half);          // columns cg .. cg + 15 of the atom
        float v[16];
        tmem_ld16(taddr + (uint32_t)cg, v);
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
            __half h0, l0, h1, l1;
            split_h(v[q] * sc, h0, l0);
            split_h(v[q + 1] * sc, h1, l1);
            const uint32_t off = atom_off(row, cg + q);
            *reinterpret_cast<__half2 *>(a + off) = __halves2half2(h0, h1);
            *reinterpret_cast<__half2 *>(a + 128 * 128 + off) = __halves2half2(l0, l1);
        }
    }
}

// Sky strips written beside the pixels (forward, hour-angle form): value v of pixel (d, r) goes
// to hi/lo[d Ly + r q] as the 16-bit hi / lo parts of sc v; hi == nullptr: none.
struct StripOut {
    uint16_t *hi, *lo;         // channel's strips, offset to the element of pixel 0
    int Ly, q, bf16;
    int vec4;                  // q == 1 and every row's element of pixel 0 8-byte aligned
    float sc;
};

__device__ __forceinline__ uint32_t strip_split(const StripOut &so, float v, uint32_t &lo)
{
    const float y = so.sc * v;
    if (so.bf16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(y);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(y - __bfloat162float(h)));
        return __bfloat16_as_ushort(h);
    }
    const __half h = __float2half_rn(y);
    lo = __half_as_ushort(__float2half_rn(y - __half2float(h)));
    return __half_as_ushort(h);
}

__device__ __forceinline__ void strip_put(const StripOut &so, int row, int col, float v)
{
    const size_t e = (size_t)row * so.Ly + (size_t)col * so.q;
    uint32_t lo;
    so.hi[e] = (uint16_t)strip_split(so, v, lo);
    so.lo[e] = (uint16_t)lo;
}

// four consecutive pixels of a row (vec4 strips): one 8-byte store per part
__device__ __forceinline__ void strip_put4(const StripOut &so, int row, int col, const float *v)
{
    const size_t e = (size_t)row * so.Ly + (size_t)col;
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = strip_split(so, v[q], l[q]);
    *reinterpret_cast<uint2 *>(so.hi + e) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    *reinterpret_cast<uint2 *>(so.lo + e) = make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
}

// Result rows (TMEM lanes) to a row-major array out[row * ld + col], times `inv`: each warp
// passes its 32 rows x 16 columns through a shared-memory tile (32 rows of 20 floats: 16-byte
// pieces, conflict-free for the row-wise writes) so that one store instruction writes 16
// consecutive columns of eight rows (16 bytes a lane when the rows are 16-byte aligned, one
// float otherwise, two rows an instruction); rows >= nrows and columns >= ncols are skipped.
// Every stored value also goes to the strips `so` when so.hi != nullptr.  Returns the largest
// |value| this thread stored.
__device__ __forceinline__ float md_store_rows(uint32_t tmem, int c0, int cols_pad, int row_base, int nrows, int ncols,
                                               float inv, float *__restrict__ out, size_t ld, float *tile,
                                               const StripOut &so)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = w & 3, half = w >> 2;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
    const int row0 = row_base + 32 * quarter;
    float *t = tile + (size_t)w * (32 * 20);
    const bool vec = (ld & 3) == 0 && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    float mx = 0.f;
    for (int cg = 16 * half; cg < cols_pad; cg += 32) {
        float v[16];
        tmem_ld16(taddr + (uint32_t)cg, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            *reinterpret_cast<float4 *>(t + lane * 20 + 4 * k) =
                make_float4(v[4 * k] * inv, v[4 * k + 1] * inv, v[4 * k + 2] * inv, v[4 * k + 3] * inv);
        __syncwarp();
        if (vec) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rr = 8 * i + (lane >> 2), cc = 4 * (lane & 3);
                const int row = row0 + rr, col = cg + cc;
                const float4 a = *reinterpret_cast<const float4 *>(t + rr * 20 + cc);
                if (row < nrows) {
                    const float e[4] = {a.x, a.y, a.z, a.w};
                    if (col + 3 < ncols) {
                        *reinterpret_cast<float4 *>(out + (size_t)row * ld + col) = a;
                        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
                        if (so.hi) {
                            if (so.vec4) {
                                strip_put4(so, row, col, e);
                            } else {
#pragma unroll
                                for (int q = 0; q < 4; ++q) strip_put(so, row, col + q, e[q]);
                            }
                        }
                    } else {
                        for (int q = 0; q < 4; ++q)
                            if (col + q < ncols) {
                                out[(size_t)row * ld + col + q] = e[q];
                                mx = fmaxf(mx, fabsf(e[q]));
                                if (so.hi) strip_put(so, row, col + q, e[q]);
                            }
                    }
                }
            }
        } else {
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int rr = 2 * i + (lane >> 4), cc = lane & 15;
                const int row = row0 + rr, col = cg + cc;
                const float xv = t[rr * 20 + cc];
                if (row < nrows && col < ncols) {
                    out[(size_t)row * ld + col] = xv;
                    mx = fmaxf(mx, fabsf(xv));
                    if (so.hi) strip_put(so, row, col, xv);
                }
            }
        }
        __syncwarp();
    }
    return mx;
}

// largest |value| of a TMEM accumulator (all threads receive it)
__device__ __forceinline__ float md_tmem_max(uint32_t tmem, int c0, int ncols, float *red)
{
    const int w = threadIdx.x >> 5, quarter = w & 3, half = w >> 2;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
    float m = 0.f;
    for (int cg = 16 * half; cg < ncols; cg += 32) {
        float v[16];
        tmem_ld16(taddr + (uint32_t)cg, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) m = fmaxf(m, fabsf(v[q]));
    }
    return block_max(m, red);
}

// Operands of one direction's two chained products (the kernels below say which is which).
struct MdPlan {
    const uint8_t *img1;    // stage-1 A image atoms (2 x 128 rows x 128 bytes each)
    const uint8_t *img2;    // stage-2 B image atoms (2 x nb2 rows x 128 bytes each)
    const float *src;       // stage-1 B operand, row-major [src_rows][src_cols]
    int src_rows, src_cols;
    int n1;                 // stage-1 K atoms
    int nb1;                // stage-1 N (rows of its B atoms, padded) = stage-2 K
    int nb2;                // stage-2 N
    bool skip_dc;           // read src[0][0] as zero
};

__device__ __forceinline__ uint32_t md_setup(const MdSmem &m, int ncols)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(m.bar_img(s), 1);
            mbar_init(m.bar_mma(s), 1);
        }
        *m.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) tmem_alloc(su32(m.tmem_slot), (uint32_t)ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *m.tmem_slot;
}

// Both products of one CTA through `ns` operand slots.  Atom i (stage 1 for i < n1, stage 2
// after) uses slot i % ns.  Its basis-image part arrives by one bulk copy, issued by thread 0
// as soon as the slot's previous atom (i - ns) has been read by its MMAs (the first ns at
// once, while the CTA scans the FP32 operand for its scale); its other part is written by
// all threads: in stage 1 the FP32 operand split into FP16 hi/lo, in stage 2 the first
// product read from TMEM, scaled and split.  Thread 0 issues each atom's 12 MMAs and commits
// them to the slot's barrier without waiting, so that filling atom i + 1 overlaps the MMAs
// of atom i.  The first product occupies TMEM columns 0 .. nb1, the second nb1 .. nb1 + nb2.
// sa and g are the power-of-two scales of the two products' B and A operands.  Returns false
// after a timeout (abort flag raised; the copies and MMAs in flight drained).
__device__ __forceinline__ bool md_two_stage(const MdSmem &m, int ns, uint32_t tmem, const MdPlan &p, float &sa,
                                             float &g)
{
    const int tid = threadIdx.x;
    const int n = p.n1 + p.nb1 / 64;
    auto slot = [&](int j) { return ns == 2 ? (j & 1) : 0; };
    auto par = [&](int j) { return (uint32_t)((j / ns) & 1); };   // phase of atom j on its slot's barriers
    const uint32_t b2_bytes = 2u * (uint32_t)p.nb2 * 128u;
    auto img_issue = [&](int i) {
        const int s = slot(i);
        if (i < p.n1) {
            mbar_expect_tx(m.bar_img(s), 2u * 128u * 128u);
            bulk_g2s(m.a_s(s), p.img1 + (size_t)i * 2 * 128 * 128, 2u * 128u * 128u, m.bar_img(s));
        } else {
            mbar_expect_tx(m.bar_img(s), b2_bytes);
            bulk_g2s(m.b_s(s), p.img2 + (size_t)(i - p.n1) * b2_bytes, b2_bytes, m.bar_img(s));
        }
    };
    // thread 0: the last atom whose image copy / MMAs it issued, per slot
    int last_img0 = -1, last_img1 = -1, last_mma0 = -1, last_mma1 = -1;
    if (tid == 0)
        for (int i = 0; i < ns && i < n; ++i) {
            img_issue(i);
            (i == 0 ? last_img0 : last_img1) = i;
        }
    sa = pow2_below(md_absmax(p.src, p.src_rows, p.src_cols, p.skip_dc, m.red));
    g = 1.f;
    const uint32_t idesc1 = idesc_f16(128, p.nb1, 0), idesc2 = idesc_f16(128, p.nb2, 0);
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        const int s = slot(i);
        if (i >= ns) {                          // the slot's previous atom is consumed
            mbar_wait_ab<32>(m.bar_mma(s), par(i - ns), m.abort_flag);
            if (tid == 0 && *m.abort_flag == 0) {
                img_issue(i);
                (s == 0 ? last_img0 : last_img1) = i;
            }
        }
        if (i == p.n1)                          // the first product is complete
            mbar_wait_ab<32>(m.bar_mma(slot(p.n1 - 1)), par(p.n1 - 1), m.abort_flag);
        __syncthreads();
        if (*m.abort_flag) {
            ok = false;
            break;
        }
        if (i < p.n1) {
            md_convert_atom(p.src, p.src_rows, p.src_cols, p.nb1, i, sa, p.skip_dc, m.b(s));
        } else {
            if (i == p.n1) {
                tc_fence_after();
                g = pow2_below(md_tmem_max(tmem, 0, p.nb1, m.red));
            }
            md_tmem_to_atom(tmem, 0, i - p.n1, g, m.a(s));
            tc_fence_before();
        }
        md_filled();
        if (tid == 0 && mbar_wait_ab<32>(m.bar_img(s), par(i), m.abort_flag)) {
            tc_fence_after();
            if (i < p.n1) issue_atom(tmem, m.a_s(s), m.b_s(s), p.nb1, i == 0, idesc1);
            else issue_atom(tmem + (uint32_t)p.nb1, m.a_s(s), m.b_s(s), p.nb2, i == p.n1, idesc2);
            mma_commit(m.bar_mma(s));
            (s == 0 ? last_mma0 : last_mma1) = i;
        }
    }
    if (ok) mbar_wait_ab<32>(m.bar_mma(slot(n - 1)), par(n - 1), m.abort_flag);   // all MMAs
    tc_fence_after();
    __syncthreads();
    if (*m.abort_flag) {
        ok = false;
        if (tid == 0) {
            if (last_img0 >= 0) mbar_drain(m.bar_img(0), par(last_img0));
            if (last_img1 >= 0) mbar_drain(m.bar_img(1), par(last_img1));
            if (last_mma0 >= 0) mbar_drain(m.bar_mma(0), par(last_mma0));
            if (last_mma1 >= 0) mbar_drain(m.bar_mma(1), par(last_mma1));
        }
        __syncthreads();
    }
    return ok;
}

__device__ __forceinline__ void md_finish(const MdSmem &m, bool ok, int *status, uint32_t tmem, int ncols)
{
    tc_fence_before();
    __syncthreads();
    if (!ok && threadIdx.x == 0) atomicExch(status, (int)FM_ERR_TIMEOUT);
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)ncols);
    }
}

// ---------------------------------------------------------------- forward
// CTA (f, d tile): stage 1 D1[d][m] = Leg_tile a_f^T over n (A = Leg tile image, B = a_f
// rows m); stage 2 D2[d][r] = W Phi^T over m (A = scaled W from TMEM, B = Phi image);
// x[f][d][r] = D2 / scales.  xmax != NULL: the largest |x| the CTA wrote goes to xmax[f] by
// atomicMax on its float bits (non-negative floats order like their bit patterns, so the
// result is independent of order).
__global__ void __launch_bounds__(MD_THREADS, 1)
k_modes_fwd(MdDims z, int ns, const float *__restrict__ a_all, int skip_dc, const uint8_t *__restrict__ leg_img,
            const uint8_t *__restrict__ phi_img, float *__restrict__ x_all, int *__restrict__ status, int ncols,
            unsigned *__restrict__ xmax, StripArgs sp)
{
    const int f = blockIdx.x, dt = blockIdx.y;
    const MdSmem m = md_smem(z.Mp > z.Rp ? z.Mp : z.Rp, ns);
    const uint32_t tmem = md_setup(m, ncols);
    MdPlan p;
    p.img1 = leg_img + (size_t)dt * (z.Np / 64) * 2 * 128 * 128;
    p.img2 = phi_img;
    p.src = a_all + (size_t)f * z.M * z.N;
    p.src_rows = z.M;
    p.src_cols = z.N;
    p.n1 = z.Np / 64;
    p.nb1 = z.Mp;
    p.nb2 = z.Rp;
    p.skip_dc = skip_dc != 0;
    float sa, g;
    const bool ok = md_two_stage(m, ns, tmem, p, sa, g);
    // x = D2 / (g 2^28 sa), through slot 0's A atom (free once the last MMAs are complete);
    // with strips (one CTA per channel) the channel's largest |x| is read from TMEM first
    // (inv is a power of two, so it is the largest stored |x| exactly) and sets their scale
    const float inv = 1.f / (g * MD_CSCALE * MD_CSCALE * sa);
    StripOut so{nullptr, nullptr, 0, 1, 0, 0, 1.f};
    if (sp.hi && ok) {                          // uniform
        const float cm = md_tmem_max(tmem, z.Mp, z.Rp, m.red) * inv;
        so.hi = sp.hi + (size_t)f * z.D * sp.Ly + sp.off;
        so.lo = sp.lo + (size_t)f * z.D * sp.Ly + sp.off;
        so.Ly = sp.Ly;
        so.q = sp.q;
        so.bf16 = sp.bf16;
        so.vec4 = sp.q == 1 && (sp.off & 3) == 0 && (sp.Ly & 3) == 0 &&
                  ((reinterpret_cast<uintptr_t>(sp.hi) | reinterpret_cast<uintptr_t>(sp.lo)) & 7) == 0;
        so.sc = pow2_below(cm);
        if (threadIdx.x == 0) xmax[f] = __float_as_uint(cm);
    }
    float xm = 0.f;
    if (ok)
        xm = md_store_rows(tmem, z.Mp, z.Rp, 128 * dt, z.D, z.R, inv, x_all + (size_t)f * z.D * z.R, (size_t)z.R,
                           reinterpret_cast<float *>(m.a(0)), so);
    if (xmax && !sp.hi) {                       // uniform: every thread takes part
        const float bm = block_max(xm, m.red);
        if (threadIdx.x == 0 && ok) atomicMax(xmax + f, __float_as_uint(bm));
    }
    md_finish(m, ok, status, tmem, ncols);
}

// ---------------------------------------------------------------- adjoint
// CTA (f, m tile): stage 1 D1[m][d] = PhiT_tile xbar_f^T over r (A = PhiT tile image, B =
// xbar_f rows d); stage 2 D2[m][n] = U LegT^T over d (A = scaled U from TMEM, B = LegT
// image); abar = D2 / scales.
__global__ void __launch_bounds__(MD_THREADS, 1)
k_modes_adj(MdDims z, int ns, const float *__restrict__ xb_all, const uint8_t *__restrict__ phit_img,
            const uint8_t *__restrict__ legt_img, float *__restrict__ abar_all, int *__restrict__ status, int ncols)
{
    const int f = blockIdx.x, mtile = blockIdx.y;
    const MdSmem m = md_smem(z.Dp > z.Np ? z.Dp : z.Np, ns);
    const uint32_t tmem = md_setup(m, ncols);
    MdPlan p;
    p.img1 = phit_img + (size_t)mtile * (z.Rp / 64) * 2 * 128 * 128;
    p.img2 = legt_img;
    p.src = xb_all + (size_t)f * z.D * z.R;
    p.src_rows = z.D;
    p.src_cols = z.R;
    p.n1 = z.Rp / 64;
    p.nb1 = z.Dp;
    p.nb2 = z.Np;
    p.skip_dc = false;
    float sx, g;
    const bool ok = md_two_stage(m, ns, tmem, p, sx, g);
    if (ok) {
        const float inv = 1.f / (g * MD_CSCALE * MD_CSCALE * sx);
        md_store_rows(tmem, z.Dp, z.Np, 128 * mtile, z.M, z.N, inv, abar_all + (size_t)f * z.M * z.N, (size_t)z.N,
                      reinterpret_cast<float *>(m.a(0)), StripOut{nullptr, nullptr, 0, 1, 0, 0, 1.f});
    }
    md_finish(m, ok, status, tmem, ncols);
}

MdDims md_dims(const Ctx &c)
{
    MdDims z;
    z.F = c.F; z.M = c.M; z.N = c.N; z.R = c.R; z.D = c.D;
    z.Mp = (c.M + 63) / 64 * 64; z.Np = (c.N + 63) / 64 * 64;
    z.Rp = (c.R + 63) / 64 * 64; z.Dp = (c.D + 63) / 64 * 64;
    return z;
}

size_t md_smem_bytes(int b_rows_max, int ns) { return 1024 + (size_t)ns * md_slot_bytes(b_rows_max) + 128; }

// two operand slots when the grid fills at most one wave of one CTA per SM; one otherwise
// (smaller CTAs: two can share an SM where TMEM allows)
int md_slots(int grid)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return grid <= sms ? 2 : 1;
}

int md_cols(int n)
{
    int c = 32;
    while (c < n) c *= 2;
    return c;
}

}  // namespace

// Images of the basis tables (once per handle) and the on/off decision: the tensor-core
// transforms run for the split-precision handles when every padded dimension is at most
// 256 (one MMA N, two TMEM accumulators within 512 columns).
fm_status modes_tc_setup(Ctx &c)
{
    ModesTc &s = c.mtc;
    s.on = false;
    if (c.prec < FM_PREC_BF16X1) return FM_OK;
    if (const char *e = getenv("FM_MODES_TC"))
        if (atoi(e) == 0) return FM_OK;
    const MdDims z = md_dims(c);
    if (z.Mp > 256 || z.Np > 256 || z.Rp > 256 || z.Dp > 256) return FM_OK;
    const int ndt = (c.D + 127) / 128, nmt = (c.M + 127) / 128;
    const size_t leg_n = (size_t)ndt * 2 * 128 * z.Np, phi_n = 2 * (size_t)z.Rp * z.Mp;
    const size_t phit_n = (size_t)nmt * 2 * 128 * z.Rp, legt_n = 2 * (size_t)z.Np * z.Dp;
    uint8_t *buf = nullptr;
    FM_CK(cudaMalloc(&buf, 2 * (leg_n + phi_n + phit_n + legt_n)));
    c.allocs.push_back(buf);
    s.leg_img = buf;
    s.phi_img = s.leg_img + 2 * leg_n;
    s.phit_img = s.phi_img + 2 * phi_n;
    s.legt_img = s.phit_img + 2 * phit_n;
    for (int dt = 0; dt < ndt; ++dt) {
        k_md_image<<<256, 256>>>(c.g.leg64, c.D, c.N, 0, 128 * dt, 128, z.Np, MD_CSCALE,
                                 s.leg_img + (size_t)dt * 2 * 2 * 128 * z.Np);
        FM_CK_LAUNCH();
    }
    k_md_image<<<256, 256>>>(c.g.phi64, c.R, c.M, 0, 0, z.Rp, z.Mp, MD_CSCALE, s.phi_img);
    FM_CK_LAUNCH();
    for (int mt = 0; mt < nmt; ++mt) {
        k_md_image<<<256, 256>>>(c.g.phi64, c.R, c.M, 1, 128 * mt, 128, z.Rp, MD_CSCALE,
                                 s.phit_img + (size_t)mt * 2 * 2 * 128 * z.Rp);
        FM_CK_LAUNCH();
    }
    k_md_image<<<256, 256>>>(c.g.leg64, c.D, c.N, 1, 0, z.Np, z.Dp, MD_CSCALE, s.legt_img);
    FM_CK_LAUNCH();
    FM_CK(smem_opt_in(k_modes_fwd));
    FM_CK(smem_opt_in(k_modes_adj));
    FM_CK(cudaDeviceSynchronize());
    s.on = true;
    return FM_OK;
}

fm_status launch_modes_tc_forward(Ctx &c, const float *a, float *x, cudaStream_t st, int skip_dc, unsigned *xmax,
                                  const StripArgs *strips)
{
    const MdDims z = md_dims(c);
    const int ndt = (c.D + 127) / 128, ns = md_slots(c.F * ndt);
    if (strips && (ndt != 1 || !xmax)) {
        set_error("sky strips need one CTA per channel and the channel maxima");
        return FM_ERR_STATE;
    }
    k_modes_fwd<<<dim3(c.F, ndt), MD_THREADS, md_smem_bytes(z.Mp > z.Rp ? z.Mp : z.Rp, ns), st>>>(
        z, ns, a, skip_dc, c.mtc.leg_img, c.mtc.phi_img, x, c.status, md_cols(z.Mp + z.Rp), xmax,
        strips ? *strips : StripArgs{});
    FM_CK_LAUNCH();
    return FM_OK;
}

fm_status launch_modes_tc_adjoint(Ctx &c, const float *xbar, float *abar, cudaStream_t st)
{
    return launch_modes_tc_adjoint_maps(c, xbar, c.F, abar, st);
}

// the same transform for nmaps pixel maps xbar[nmaps][D][R] -> abar[nmaps][M][N]
fm_status launch_modes_tc_adjoint_maps(Ctx &c, const float *xbar, int nmaps, float *abar, cudaStream_t st)
{
    MdDims z = md_dims(c);
    z.F = nmaps;
    const int nmt = (c.M + 127) / 128, ns = md_slots(nmaps * nmt);
    k_modes_adj<<<dim3(nmaps, nmt), MD_THREADS, md_smem_bytes(z.Dp > z.Np ? z.Dp : z.Np, ns), st>>>(
        z, ns, xbar, c.mtc.phit_img, c.mtc.legt_img, abar, c.status, md_cols(z.Dp + z.Np));
    FM_CK_LAUNCH();
    return FM_OK;
}

}  // namespace fm
