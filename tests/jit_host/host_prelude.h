// Host build of the part kernels that the library generates for a plan
// (test infrastructure only: the library never runs this). The generated
// CUDA source of a part uses a small set of helpers (copies, stores, packed
// float pairs, register permutations) from the run-time prelude; this header
// gives each of them the same meaning in plain C++, and the CUDA thread
// model (threadIdx, __syncthreads, dynamic shared memory) is emulated with
// one std::thread per CUDA thread of a single CTA and a std::barrier. A test
// compiles the generated source of every part with g++ against this header
// and compares the resulting state with the oracle, so that the generator's
// layouts and straight-line arithmetic are checked without a GPU.
#pragma once
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstring>

#define __device__
#define __global__
#define __forceinline__ inline
#define __restrict__
#define __launch_bounds__(a, b)
#define __align__(n) __attribute__((aligned(n)))
#define __shared__
#define HISV_HOST_SMEM_BYTES (2u << 20)

struct hisv_dim3 { unsigned x = 0, y = 0, z = 0; };
inline thread_local hisv_dim3 threadIdx;
inline hisv_dim3 blockIdx;
inline hisv_dim3 gridDim{1, 1, 1};
inline std::barrier<> *hisv_host_barrier = nullptr;
inline void __syncthreads() { hisv_host_barrier->arrive_and_wait(); }
alignas(16) inline unsigned char smem_raw[HISV_HOST_SMEM_BYTES];

struct float2 { float x, y; };
struct double2 { double x, y; };
inline float2 make_float2(float x, float y) { return float2{x, y}; }

#include "ops_core.cuh"

namespace hisv {

#if HISV_DF
struct df {
    float hi, lo;
    df() = default;
    constexpr df(float h, float l) : hi(h), lo(l) {}
    df(int v) : hi((float)v), lo(0.f) {}
};
inline df df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return df(s, b - (s - a));
}
inline df operator+(df a, df b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_fast_two_sum(s, e + (a.lo + b.lo));
}
inline df operator-(df a) { return df(-a.hi, -a.lo); }
inline df operator-(df a, df b) { return a + (-b); }
inline df operator*(df a, df b) {
    const float p = a.hi * b.hi;
    float e = std::fmaf(a.hi, b.hi, -p);
    e = std::fmaf(a.hi, b.lo, e);
    e = std::fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
struct alignas(16) cdf { df x, y; };
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

// copies complete at once on the host; the kernels' double buffering and
// barriers keep the same order of reads and writes
inline void cp_async(void *smem, const void *gmem) { std::memcpy(smem, gmem, sizeof(C)); }
inline void cp_commit() {}
inline void cp_wait1() {}
inline void cp_wait0() {}
inline void st_amp(C *p, const C &v) { *p = v; }

inline u64 deposit64(u64 v, u64 mask) {
    u64 out = 0;
    for (int b = 0; b < 64; b++)
        if ((mask >> b) & 1) {
            if (v & 1) out |= 1ull << b;
            v >>= 1;
        }
    return out;
}

#if !HISV_FP64 && !HISV_DF
inline float2 add2(float2 a, float2 b) { return float2{a.x + b.x, a.y + b.y}; }
inline float2 sub2(float2 a, float2 b) { return float2{a.x - b.x, a.y - b.y}; }
inline float2 fma2(float t, float2 b, float2 c) { return float2{std::fmaf(t, b.x, c.x), std::fmaf(t, b.y, c.y)}; }
template <int B>
inline void op_h2(C (&a)[NR]) {
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i] = add2(x, y);
        a[j] = sub2(x, y);
    }
}
template <int B, int F>
inline void op_rys2(C (&a)[NR], float t) {
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        if (F == 0) {
            a[i] = fma2(-t, y, x);
            a[j] = fma2(t, x, y);
        } else {
            a[i] = fma2(t, x, make_float2(-y.x, -y.y));
            a[j] = fma2(t, y, x);
        }
    }
}
#endif

template <int B>
inline void op_x(C (&a)[NR]) {
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const C t = a[i];
        a[i] = a[i | (1 << B)];
        a[i | (1 << B)] = t;
    }
}
template <int B>
inline void op_y(C (&a)[NR]) {
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
template <int A, int B>
inline void op_cx(C (&a)[NR]) {
    for (int i = 0; i < NR; i++) {
        if (!(i & (1 << A)) || (i & (1 << B))) continue;
        const C t = a[i];
        a[i] = a[i | (1 << B)];
        a[i | (1 << B)] = t;
    }
}
template <int B>
inline void op_cxt(C (&a)[NR], bool ctl) {
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i] = ctl ? y : x;
        a[j] = ctl ? x : y;
    }
}
template <int B>
inline void op_sgn(C (&a)[NR], bool neg) {
    for (int i = 0; i < NR; i++)
        if ((i & (1 << B)) && neg) { a[i].x = -a[i].x; a[i].y = -a[i].y; }
}
inline void tmul(Real &tpr, Real &tpi, Real dr, Real di) {
    const Real x = tpr, y = tpi;
    tpr = x * dr - y * di;
    tpi = x * di + y * dr;
}

}  // namespace hisv
