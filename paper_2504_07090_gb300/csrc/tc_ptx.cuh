// Inline-PTX wrappers for the sm_103a tensor-core kernels: mbarriers (bounded waits),
// TMEM allocation, tcgen05.mma / commit / ld, shared-memory matrix descriptors for the
// 128-byte-swizzled K-major layout, bulk copies, and the FP16 / BF16 hi-lo operand split.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fm {
namespace tc {

constexpr long long WAIT_CYCLES = 4000000000LL;       // ~2 s at 2 GHz
// upper bound on how long a waiting thread may stay suspended inside one try_wait
// (it resumes as soon as the phase completes); keeps idle waiters off the issue slots
constexpr uint32_t SUSPEND_NS = 1000000u;

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(bar) : "memory");
}

// bounded wait that also gives up when another warp raised the CTA's abort flag;
// SLEEP_NS > 0 backs off between polls (for roles that mostly wait: the MMA issuer,
// the bulk-copy issuer and the epilogue), keeping the issue slots for the producers
template <int SLEEP_NS = 0>
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                             long long limit = WAIT_CYCLES)
{
    long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(SUSPEND_NS)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            return false;
        }
        if (SLEEP_NS > 0) __nanosleep(SLEEP_NS);
    }
}

// bounded wait that ignores the abort flag (draining copies or MMAs before exit)
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity)
{
    long long t0 = clock64();
    while (clock64() - t0 < WAIT_CYCLES) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(SUSPEND_NS)
            : "memory");
        if (ok) return;
    }
}

// arrive once and add `bytes` to the transaction count the phase waits for
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing `bytes` transactions on mbarrier `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// named barrier `id` over `nthreads` threads; returns the OR of every thread's `pred`
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool pred)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred q, p;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(out)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return out != 0;
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

// D[tmem] (+)= A[tmem] * B[smem]^T: A (M rows on the TMEM lanes, two 16-bit K elements per
// 32-bit column, lower K in the low half) read from tensor memory, FP32 accumulate
__device__ __forceinline__ void mma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc)
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

// 32 lanes x 16 consecutive 32-bit columns, register -> TMEM
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 32 lanes x 8 consecutive 32-bit columns, register -> TMEM (completion: tmem_wait_st)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 lanes x 16 columns, register -> TMEM (completion: tmem_wait_st): thread t writes lanes
// t / 4 (r[0], r[1], r[4], r[5]) and t / 4 + 8 (r[2], r[3], r[6], r[7]) of the 16 starting at
// taddr's lane, columns 2 (t % 4) + {0, 1} (r[0..3]) and 8 + 2 (t % 4) + {0, 1} (r[4..7])
__device__ __forceinline__ void tmem_st_16x256b_x2(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// Shared-memory matrix descriptor, K-major without swizzle: 8 x 16-byte core matrices stored
// as 128 contiguous bytes; `lbo` = byte step between core matrices adjacent in K, `sbo` =
// byte step between 8-row groups (both multiples of 16).
__device__ __forceinline__ uint64_t sdesc_none(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;                           // descriptor version for tcgen05; swizzle 0 = none
    return d;
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
    // v = (low, high) element of one packed column; the residual in one packed FMA
    static __device__ __forceinline__ void split2(float2 v, uint32_t &hi, uint32_t &lo)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        const float2 r = __ffma2_rn(__bfloat1622float2(h), make_float2(-1.f, -1.f), v);
        __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
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
    static __device__ __forceinline__ void split2(float2 v, uint32_t &hi, uint32_t &lo)
    {
        __half2 h = __floats2half2_rn(v.x, v.y);
        const float2 r = __ffma2_rn(__half22float2(h), make_float2(-1.f, -1.f), v);
        __half2 l = __floats2half2_rn(r.x, r.y);
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


}  // namespace tc
}  // namespace fm
