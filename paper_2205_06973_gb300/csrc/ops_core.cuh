// Register-level gate arithmetic on a thread's 2^R amplitudes, with
// compile-time register bits. Self-contained (no standard or CUDA headers),
// so that both the library's kernels and the part kernels compiled for a
// plan at run time (NVRTC) use the same definitions.
//
// A thread holds 2^R amplitudes a[0..2^R) of its tile; register bit b of the
// index i is one tile slot (qubit).
#pragma once

namespace hisv {

// ------------------------------------------------------------------------
// register-bit operations; B, A are compile-time register bits
// ------------------------------------------------------------------------
// Hadamard without its 1/sqrt2: the planner folds the factor into the part's
// store factor, so each H costs one add and one subtract per amplitude pair.
template <int NR, int B, typename C>
__device__ __forceinline__ void op_h(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i].x = x.x + y.x; a[i].y = x.y + y.y;
        a[j].x = x.x - y.x; a[j].y = x.y - y.y;
    }
}

template <int NR, int B, typename C, typename Real>
__device__ __forceinline__ void op_u2(C (&a)[NR], const Real *m) {
    const Real m00r = m[0], m00i = m[1], m01r = m[2], m01i = m[3];
    const Real m10r = m[4], m10i = m[5], m11r = m[6], m11i = m[7];
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i].x = m00r * x.x - m00i * x.y + m01r * y.x - m01i * y.y;
        a[i].y = m00r * x.y + m00i * x.x + m01r * y.y + m01i * y.x;
        a[j].x = m10r * x.x - m10i * x.y + m11r * y.x - m11i * y.y;
        a[j].y = m10r * x.y + m10i * x.x + m11r * y.y + m11i * y.x;
    }
}

template <int NR, int B, typename C, typename Real>
__device__ __forceinline__ void op_rx(C (&a)[NR], Real c, Real s) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i].x = c * x.x + s * y.y; a[i].y = c * x.y - s * y.x;
        a[j].x = s * x.y + c * y.x; a[j].y = c * y.y - s * x.x;
    }
}

template <int NR, int B, typename C, typename Real>
__device__ __forceinline__ void op_ry(C (&a)[NR], Real c, Real s) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        a[i].x = c * x.x - s * y.x; a[i].y = c * x.y - s * y.y;
        a[j].x = s * x.x + c * y.x; a[j].y = s * x.y + c * y.y;
    }
}

// Scaled rotations: the gate divided by its largest entry (the factor is
// applied once, with the part's store factor), so every output component is
// one multiply-add. F = form (see OP_RXS / OP_RYS / OP_U2S in program.hpp).
template <int NR, int B, int F, typename C, typename Real>
__device__ __forceinline__ void op_rxs(C (&a)[NR], Real t) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        if (F == 0) {            // (x + (-it) y, y + (-it) x)
            a[i].x = x.x + t * y.y; a[i].y = x.y - t * y.x;
            a[j].x = y.x + t * x.y; a[j].y = y.y - t * x.x;
        } else {                 // (y + (it) x, x + (it) y)
            a[i].x = y.x - t * x.y; a[i].y = y.y + t * x.x;
            a[j].x = x.x - t * y.y; a[j].y = x.y + t * y.x;
        }
    }
}

template <int NR, int B, int F, typename C, typename Real>
__device__ __forceinline__ void op_rys(C (&a)[NR], Real t) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        if (F == 0) {            // (x - t y, y + t x)
            a[i].x = x.x - t * y.x; a[i].y = x.y - t * y.y;
            a[j].x = y.x + t * x.x; a[j].y = y.y + t * x.y;
        } else {                 // (t x - y, x + t y)
            a[i].x = t * x.x - y.x; a[i].y = t * x.y - y.y;
            a[j].x = x.x + t * y.x; a[j].y = x.y + t * y.y;
        }
    }
}

template <int NR, int B, int F, typename C, typename Real>
__device__ __forceinline__ void op_u2s(C (&a)[NR], Real ur, Real ui, Real vr, Real vi, Real wr, Real wi) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) continue;
        const int j = i | (1 << B);
        const C x = a[i], y = a[j];
        if (F == 0) {            // (x + u y, v x + w y)
            a[i].x = x.x + ur * y.x - ui * y.y; a[i].y = x.y + ur * y.y + ui * y.x;
        } else {                 // (u x + y, v x + w y)
            a[i].x = y.x + ur * x.x - ui * x.y; a[i].y = y.y + ur * x.y + ui * x.x;
        }
        a[j].x = vr * x.x - vi * x.y + wr * y.x - wi * y.y;
        a[j].y = vr * x.y + vi * x.x + wr * y.y + wi * y.x;
    }
}

template <typename C, typename Real>
__device__ __forceinline__ void cmul_in(C &v, Real dr, Real di) {
    const Real x = v.x, y = v.y;
    v.x = x * dr - y * di;
    v.y = x * di + y * dr;
}

template <int NR, int B, typename C, typename Real>
__device__ __forceinline__ void op_d(C (&a)[NR], Real d0r, Real d0i, Real d1r, Real d1i) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        if (i & (1 << B)) cmul_in(a[i], d1r, d1i);
        else cmul_in(a[i], d0r, d0i);
    }
}

template <int NR, int B, typename C, typename Real>
__device__ __forceinline__ void op_p(C (&a)[NR], Real dr, Real di) {
#pragma unroll
    for (int i = 0; i < NR; i++)
        if (i & (1 << B)) cmul_in(a[i], dr, di);
}

template <int NR, int B, typename C>
__device__ __forceinline__ void op_z(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++)
        if (i & (1 << B)) { a[i].x = -a[i].x; a[i].y = -a[i].y; }
}

template <int NR, int A, int B, typename C, typename Real>
__device__ __forceinline__ void op_cp(C (&a)[NR], Real dr, Real di) {
#pragma unroll
    for (int i = 0; i < NR; i++)
        if ((i & (1 << A)) && (i & (1 << B))) cmul_in(a[i], dr, di);
}

template <int NR, int A, int B, typename C>
__device__ __forceinline__ void op_cz(C (&a)[NR]) {
#pragma unroll
    for (int i = 0; i < NR; i++)
        if ((i & (1 << A)) && (i & (1 << B))) { a[i].x = -a[i].x; a[i].y = -a[i].y; }
}

// Swizzled shared-memory index contribution of tile slot p. The swizzle XORs
// the slot bits above the bank group into the low bits (linear over GF(2)),
// so a warp whose lane bits sit on slots of distinct residues touches
// distinct banks: 8-byte elements use 4-bit groups, 16-byte elements 3-bit.
template <typename Real>
__device__ __forceinline__ unsigned int swz(int p) {
    if constexpr (sizeof(Real) == 4) return p < 4 ? (1u << p) : ((1u << p) | (1u << (p & 3)));
    else return p < 3 ? (1u << p) : ((1u << p) | (1u << (p % 3)));
}


}  // namespace hisv
