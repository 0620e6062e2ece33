// Prelude of the part kernels that are generated for one plan and compiled
// at run time (NVRTC, sm_103a). Self-contained: only ops_core.cuh, which the
// library hands to the compiler as an in-memory header. HISV_FP64 selects
// complex128 (1) or complex64 (0) amplitudes, HISV_DF = 1 complex128 held as
// double-float pairs; HISV_R the register bits per thread.
//
// A generated kernel is the part kernel of Algorithm 1 (Gather - Execute -
// Scatter) with everything known at plan time folded in: the tile's qubits
// and outer mask, the register phases' shared-memory layouts, and each gate
// as straight-line code on compile-time register indices with its
// coefficients as literals. Register permutations (X, Y, CX on register
// bits) become renamings, which cost nothing in straight-line code.
#pragma once
#include "ops_core.cuh"

namespace hisv {

#if HISV_DF
// Double-float arithmetic: a real is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2 (about 48 significant bits; Dekker 1971).
// Sums use Knuth's error-free TwoSum of the high parts (TAOCP vol. 2, 4.2.2)
// plus the low parts, renormalised by Dekker's FastTwoSum; products use the
// error-free product of the high parts through one FMA, plus the cross terms.
// The absolute error of an operation stays within a few units of 2^-48 of
// its operands' magnitude.
struct df {
    float hi, lo;
    df() = default;
    __device__ __forceinline__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ df(int v) : hi((float)v), lo(0.f) {}
};
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return df(s, b - (s - a));
}
__device__ __forceinline__ df operator+(df a, df b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_fast_two_sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
struct __align__(16) cdf {
    df x, y;
};
typedef df Real;
typedef cdf C;
#elif HISV_FP64
typedef double Real;
typedef double2 C;
#else
typedef float Real;
typedef float2 C;
#endif
typedef unsigned long long u64;
typedef unsigned int u32;
constexpr int NR = 1 << HISV_R;

__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const u32 s = (u32)__cvta_generic_to_shared(smem);
    if (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Streaming (evict-first) store of one amplitude.
__device__ __forceinline__ void st_amp(C *p, const C &v) {
#if HISV_DF
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo));
#else
    __stcs(p, v);
#endif
}

// Deposit the bits of v, lowest first, into the set bits of mask.
__device__ __forceinline__ u64 deposit64(u64 v, u64 mask) {
    u64 out = 0;
    while (mask) {
        const u64 low = mask & (~mask + 1);
        if (v & 1) out |= low;
        v >>= 1;
        mask ^= low;
    }
    return out;
}

#if !HISV_FP64 && !HISV_DF
// Packed pairs of floats (sm_100+ f32x2 arithmetic): a complex64 amplitude is
// one 64-bit register pair, so a complex sum or a real-scaled complex
// multiply-add is one instruction.
__device__ __forceinline__ unsigned long long pk(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
// t * b + c with the real t on both halves
__device__ __forceinline__ float2 fma2(float t, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(make_float2(t, t))), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
// H without its 1/sqrt2 (x + y, x - y) and the scaled RY, packed.
template <int B>
__device__ __forceinline__ void op_h2(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i] = add2(x, y);
        a[j] = sub2(x, y);
    }
}
template <int B, int F>
__device__ __forceinline__ void op_rys2(C (&a)[NR], float t) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        if (F == 0) {            // (x - t y, y + t x)
            a[i] = fma2(-t, y, x);
            a[j] = fma2(t, x, y);
        } else {                 // (t x - y, x + t y)
            a[i] = fma2(t, x, make_float2(-y.x, -y.y));
            a[j] = fma2(t, y, x);
        }
    }
}
#endif

// X on register bit B: exchange the halves (a renaming).
template <int B>
__device__ __forceinline__ void op_x(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const C t = a[i];
        a[i] = a[i | (1 << B)];
        a[i | (1 << B)] = t;
    }
}
// Y = [[0, -i], [i, 0]] on register bit B.
template <int B>
__device__ __forceinline__ void op_y(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i].x = y.y;
        a[i].y = -y.x;
        a[j].x = -x.y;
        a[j].y = x.x;
    }
}
// CX with control register bit A and target register bit B.
template <int A, int B>
__device__ __forceinline__ void op_cx(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (!(i & (1 << A)) || (i & (1 << B))) continue;
        const C t = a[i];
        a[i] = a[i | (1 << B)];
        a[i | (1 << B)] = t;
    }
}
// CX with its control on a thread bit (ctl) and target register bit B:
// selects, so the lanes of a warp do not diverge.
template <int B>
__device__ __forceinline__ void op_cxt(C (&a)[NR], bool ctl) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i] = ctl ? y : x;
        a[j] = ctl ? x : y;
    }
}
// The amplitudes with register bit B set are negated where neg holds (a
// controlled Z whose control is a thread bit): one packed multiply by (s, s)
// per amplitude for complex64, a multiply of each part otherwise.
template <int B>
__device__ __forceinline__ void op_sgn(C (&a)[NR], bool neg) {
#if HISV_DF
    const float s = neg ? -1.f : 1.f;
#pragma unroll
    for (int i = 0; i < NR; i++)
        if (i & (1 << B)) {
            a[i].x.hi *= s; a[i].x.lo *= s;
            a[i].y.hi *= s; a[i].y.lo *= s;
        }
#elif HISV_FP64
    const double s = neg ? -1.0 : 1.0;
#pragma unroll
    for (int i = 0; i < NR; i++)
        if (i & (1 << B)) { a[i].x *= s; a[i].y *= s; }
#else
    const float s = neg ? -1.f : 1.f;
    unsigned long long ss;
    asm("mov.b64 %0, {%1, %1};" : "=l"(ss) : "f"(s));
#pragma unroll
    for (int i = 0; i < NR; i++)
        if (i & (1 << B)) {
            unsigned long long d;
            asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a[i])), "l"(ss));
            a[i] = upk(d);
        }
#endif
}
// Per-thread phase *= (dr, di).
__device__ __forceinline__ void tmul(Real &tpr, Real &tpi, Real dr, Real di) {
    const Real x = tpr, y = tpi;
    tpr = x * dr - y * di;
    tpi = x * di + y * dr;
}

}  // namespace hisv
