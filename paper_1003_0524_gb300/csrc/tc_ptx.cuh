// tc_ptx.cuh -- inline-PTX helpers for the tensor-core kernels (sm_103a):
// mbarriers with bounded waits, TMA tile loads, tcgen05 MMA / commit / TMEM
// allocation and loads, shared-memory matrix descriptors, and the
// fixed-point slice helpers shared by every slice GEMM.
#pragma once

#include "hfx_internal.cuh"

namespace hfx {
namespace tc {

constexpr unsigned long long kWaitNs = 2000000000ULL;  // 2 s

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\tselp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok;
}
// Bounded wait.  Returns false (and raises the CTA abort flag and the global
// error word) if the phase did not complete in time or the CTA is aborting.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err,
                                          int code) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            unsigned long long now = gtimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitNs) {
                *abort_flag = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
// Bounded wait on a barrier that nothing completes, for the fault-injection
// hook of the tests: gives up after ns nanoseconds like mbar_wait does.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err,
                                             int code, unsigned long long ns) {
    unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > ns) {
            *abort_flag = 1;
            atomicCAS(err, 0, code);
            return false;
        }
    }
}
// Best-effort bounded wait used only while draining after an abort.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity)) {
        if (gtimer() - t0 > kWaitNs) return;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(dst),
        "l"((uint64_t)map), "r"(saddr(bar)), "r"(x), "r"(y)
        : "memory");
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// The MMA thread's last step: wait (bounded) until every tcgen05.mma it issued
// has completed, so that TMEM is never freed under an MMA still in flight
// (after an abort nothing else waits for them).  bar: an mbarrier of count 1
// used for nothing else.
__device__ __forceinline__ void umma_drain(uint64_t *bar) {
    umma_commit(bar);
    mbar_drain(bar, 0);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand, 128-byte swizzle:
// 8-row atoms of 1024 bytes (stride-byte-offset), leading offset unused.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// K-major operand without swizzle: core matrices of 8 rows x 16 bytes (rows
// 16 bytes apart); lbo = byte distance of the two core matrices adjacent in
// K, sbo = byte distance of core matrices adjacent in M/N.
__device__ __forceinline__ uint64_t desc_ns(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// K-major operand, 64-byte swizzle (rows of 32 BF16): 8-row atoms of 512 bytes.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// The ten kept slice products s_a t_b (a + b <= 3) fall in four weight classes
// w = a + b, one TMEM accumulator of N columns each, class w at columns w N.
// The slice planes of B sit back to back in shared memory, so the products of
// one A slice a with B slices b, b + 1, ... form one MMA of width (count) N
// whose output starts at column (a + b) N.

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}


// ------------------------------------------------------------- slices
constexpr int NPL = 4;      // slices per operand

// The slicing below runs on the integer units: GB300's FP64 pipe is far too
// narrow for a pass over every element of the projections.

// |x| as an integer that orders like |x| (non-negative doubles order like
// their bit patterns)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}

// exponent e with max < 2^e, from abs_bits(max) (0 for an all-zero line)
__device__ __forceinline__ int line_exp_bits(unsigned long long b) {
    if (b == 0) return 0;
    int E = (int)(b >> 52);
    return E == 0 ? -1021 : E - 1022;
}

// An integer d with |d| <= 256 as BF16, exactly, without conversion
// instructions: 1.5 2^23 + d has the bit pattern of 1.5 2^23 plus d (its ulp is
// 1), subtracting 1.5 2^23 leaves d exactly, and d has at most 8 significant
// bits, so the upper half of its FP32 pattern is its BF16 pattern.
__device__ __forceinline__ __nv_bfloat16 small_int_bf16(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}

// x (|x| < 2^e) as four balanced base-256 digits s_0..s_3 of
// N = round(x 2^(32-e)) (nearest, ties to even): x ~ sum_i s_i 2^(e-8(i+1)),
// |s_0| <= 256, |s_1..3| <= 128, each exact in BF16.
__device__ __forceinline__ void slice4(double x, int e, __nv_bfloat16 *o /* 4 */) {
    long long bits = __double_as_longlong(x);
    int E = (int)((bits >> 52) & 0x7ff);
    long long N = 0;
    if (E != 0) {   // zeros and subnormals give 0
        unsigned long long m = ((unsigned long long)bits & 0xfffffffffffffULL) | (1ULL << 52);
        int sh = 1043 + e - E;   // N = m 2^-sh; sh >= 21 because |x| < 2^e
        unsigned long long q = 0;
        if (sh < 64) {
            q = m >> sh;
            unsigned long long rem = m & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
            if (rem > half || (rem == half && (q & 1))) ++q;
        }
        N = bits < 0 ? -(long long)q : (long long)q;
    }
    long long d3 = ((N + 128) & 255) - 128;
    N = (N - d3) >> 8;
    long long d2 = ((N + 128) & 255) - 128;
    N = (N - d2) >> 8;
    long long d1 = ((N + 128) & 255) - 128;
    N = (N - d1) >> 8;
    o[0] = small_int_bf16((int)N);
    o[1] = small_int_bf16((int)d1);
    o[2] = small_int_bf16((int)d2);
    o[3] = small_int_bf16((int)d3);
}

// Combine the four exact class sums of one K group (units 2^(eA+eB-16)) and
// add them, scaled by sc, into the compensated pair (hi, lo).
__device__ __forceinline__ void class_accumulate(float a0, float a1, float a2, float a3, float sc, float &hi,
                                                 float &lo) {
    float c = fmaf(a3, 0x1p-8f, a2);
    c = fmaf(c, 0x1p-8f, a1);
    float x = a0 * sc;
    float s = hi + x;
    float bb = s - hi;
    float er = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += er + c * (0x1p-8f * sc);
}

// Packed FP32 pairs (two columns per instruction; each lane rounds to nearest
// exactly as the scalar operation does).
__device__ __forceinline__ uint64_t f2_pack(uint32_t x, uint32_t y) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(x), "r"(y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
    uint32_t x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(x), "=r"(y) : "l"(v));
    return make_float2(__uint_as_float(x), __uint_as_float(y));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// class_accumulate (sc = 1) for two columns at once; a_w hold the class sums
// of the two columns as packed pairs.
__device__ __forceinline__ void class_accumulate2(uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3, uint64_t &hi,
                                                  uint64_t &lo) {
    const uint64_t s8 = f2_pack(0x3b800000u, 0x3b800000u);   // 2^-8, 2^-8
    uint64_t c = f2_fma(a3, s8, a2);
    c = f2_fma(c, s8, a1);
    const uint64_t s = f2_add(hi, a0);
    const uint64_t bb = f2_sub(s, hi);
    const uint64_t er = f2_add(f2_sub(hi, f2_sub(s, bb)), f2_sub(a0, bb));
    hi = s;
    lo = f2_add(lo, f2_fma(c, s8, er));
}

// class_accumulate for two columns with per-column scales sc (packed pair)
__device__ __forceinline__ void class_accumulate2_sc(uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3, uint64_t sc,
                                                     uint64_t &hi, uint64_t &lo) {
    const uint64_t s8 = f2_pack(0x3b800000u, 0x3b800000u);   // 2^-8, 2^-8
    uint64_t c = f2_fma(a3, s8, a2);
    c = f2_fma(c, s8, a1);
    const uint64_t x = f2_mul(a0, sc);
    const uint64_t s = f2_add(hi, x);
    const uint64_t bb = f2_sub(s, hi);
    const uint64_t er = f2_add(f2_sub(hi, f2_sub(s, bb)), f2_sub(x, bb));
    hi = s;
    lo = f2_add(lo, f2_fma(c, f2_mul(s8, sc), er));
}

// x * 2^k as a double for a normal FP32 x (or zero), built from the bits of x
// with 32-bit integer operations: no FP64 conversion.  FP32 subnormals give 0.
// The scaled exponent must stay in the normal FP64 range.
__device__ __forceinline__ double f32_to_f64_scaled(float x, int k) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint32_t hi = e ? (b & 0x80000000u) | ((e + 896u + (uint32_t)k) << 20) | ((b & 0x7fffffu) >> 3) : 0u;
    const uint32_t lo = e ? b << 29 : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// (h + l) * 2^k for FP32 h, l: the two exact scaled conversions and one FP64
// add, the correctly rounded sum (exact when the exponents of h and l are
// within 29).  One FP64 operation per output: GB300's FP64 pipe is narrow, and
// the epilogues convert one value per output element.
__device__ __forceinline__ double f32pair_to_f64(float h, float l, int k) {
    return f32_to_f64_scaled(h, k) + f32_to_f64_scaled(l, k);
}

// The same value by integer operations only (no FP64 operation): both terms
// on a common 62-bit fixed point 38 bits below the larger exponent, added, and
// rounded to 53 bits, to nearest even.  Correctly rounded when the exponents
// of h and l are within 38; a smaller term further below is truncated there
// (at most one unit in the last place).  Results below the normal range give 0.
__device__ __forceinline__ double f32pair_to_f64_int(float h, float l, int k) {
    const uint32_t bh = __float_as_uint(h), bl = __float_as_uint(l);
    const int beh = (bh >> 23) & 0xff, bel = (bl >> 23) & 0xff;
    long long mh = (long long)((bh & 0x7fffffu) | (beh ? 0x800000u : 0u));
    long long ml = (long long)((bl & 0x7fffffu) | (bel ? 0x800000u : 0u));
    if (bh >> 31) mh = -mh;
    if (bl >> 31) ml = -ml;
    const int eh = (beh ? beh : 1) - 150, el = (bel ? bel : 1) - 150;   // value = m * 2^e
    const int emax = mh ? (ml ? max(eh, el) : eh) : el;
    const int e0 = emax - 38;
    const int dh = eh - e0, dl = el - e0;                                // the larger term: shift 38
    // (a signed term times 2^d as a product: left shifts of negative values are not defined)
    const long long S = (dh >= 0 ? mh * (1LL << dh) : (dh > -63 ? mh >> -dh : (mh < 0 ? -1 : 0))) +
                        (dl >= 0 ? ml * (1LL << dl) : (dl > -63 ? ml >> -dl : (ml < 0 ? -1 : 0)));
    if (S == 0) return 0.0;
    const unsigned long long sgn = S < 0 ? (1ULL << 63) : 0ULL;
    unsigned long long a = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
    const int lz = __clzll(a);
    a <<= lz;                                                           // bit 63 set
    unsigned long long m = a >> 11;                                     // 53 bits
    const unsigned long long rem = a & 0x7ffULL;
    if (rem > 0x400ULL || (rem == 0x400ULL && (m & 1ULL))) ++m;         // may carry to 2^53: exponent + 1 below
    const long long bexp = (long long)(e0 + k - lz) + 63 + 1023;        // biased exponent of the leading bit
    if (bexp < 1) return 0.0;
    return __longlong_as_double((long long)(sgn | (((unsigned long long)(bexp - 1) << 52) + m)));
}

// S + E += a * b for double-FP32 a = (ah, al), b = (bh, bl): the product's
// rounding error from an FMA, the cross terms to first order, S updated by an
// exact two-sum whose error joins E.  Relative error about 2^-46.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &S, float &E) {
    const float p = ah * bh;
    const float pe = fmaf(ah, bh, -p);
    const float cross = fmaf(ah, bl, al * bh);
    const float s = S + p;
    const float bb = s - S;
    const float err = (S - (s - bb)) + (p - bb);
    S = s;
    E += err + (pe + cross);
}

// (h, l) -> (s, e) with s = fl(h + l) and s + e = h + l exactly (two-sum)
__device__ __forceinline__ void two_sum(float h, float l, float &s, float &e) {
    s = h + l;
    const float bb = s - h;
    e = (h - (s - bb)) + (l - bb);
}

// 2^d as a float for d <= 0 (0 below the normal range)
__device__ __forceinline__ float pow2f_neg(int d) { return d >= -126 ? __int_as_float((127 + d) << 23) : 0.0f; }

int make_map_2d(hfx_ctx *ctx, CUtensorMap *m, const void *ptr, long long rows, long long cols, int box_rows);
int make_map_2d_sw(hfx_ctx *ctx, CUtensorMap *m, const void *ptr, long long rows, long long cols, int box_rows,
                   int box_cols, int swizzle_bytes);
int num_sms();

}  // namespace tc
}  // namespace hfx
