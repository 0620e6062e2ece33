// Prelude of the part kernels that are generated for one plan and compiled
// at run time (NVRTC, sm_103a). Self-contained: only ops_core.cuh, which the
// library hands to the compiler as an in-memory header. HISV_FP64 selects
// complex128 (1) or complex64 (0) amplitudes; HISV_R the register bits per
// thread.
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

#if HISV_FP64
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
// Per-thread phase *= (dr, di).
__device__ __forceinline__ void tmul(Real &tpr, Real &tpi, Real dr, Real di) {
    const Real x = tpr, y = tpi;
    tpr = x * dr - y * di;
    tpi = x * di + y * dr;
}

}  // namespace hisv
