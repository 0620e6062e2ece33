// Register-level operations of the part interpreter (shared by the part
// kernel and the batched warp-level kernel).
//
// A thread holds 2^R amplitudes a[0..2^R) of its tile; register bit b of the
// index i is one tile slot (qubit). Every op acts on compile-time register
// bits (with_bit turns a runtime bit into a template argument), so the
// amplitudes stay in registers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ops_core.cuh"
#include "program.hpp"

namespace hisv {

template <typename Real> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };

// Call f(integral_constant<int, b>) for a runtime register bit b < R.
template <int R, int B = 0, typename F>
__device__ __forceinline__ void with_bit(int b, F &&f) {
    if constexpr (B < R) {
        if (b == B) f(std::integral_constant<int, B>());
        else with_bit<R, B + 1>(b, static_cast<F &&>(f));
    }
}

// Register permutations (X, Y, CX) go through shared memory: the thread
// stores its amplitudes into its own slots of the tile buffer (slot of
// register index i: s_thr ^ XOR of s_reg[b] over the bits b of i, the
// layout the phase was loaded with) and loads them back permuted. No other
// thread touches these slots, so no barrier is needed, and no register is
// renamed inside the op switch: a permutation kept in registers renames them
// differently on every path, and reconciling those renamings at the loop's
// back edge costs every op of the interpreter (measured: about a third of
// its instructions).
// New a[i] = old a[i ^ (1 << t)] where the control holds (tctl, and bit cbit
// of i when cbit >= 0), else a[i] stays; Y also multiplies by -i (bit t of i
// clear) or +i (set).
template <int NR, int R, typename C>
__device__ __forceinline__ void perm_smem(C (&a)[NR], C *buf, uint32_t s_thr, const uint32_t (&s_reg)[R], int t,
                                          int cbit, bool tctl, bool y) {
#pragma unroll
    for (int i = 0; i < NR; i++) {
        uint32_t o = s_thr;
#pragma unroll
        for (int b = 0; b < R; b++)
            if (i & (1 << b)) o ^= s_reg[b];
        buf[o] = a[i];
    }
    uint32_t st = 0;   // s_reg[t] without a dynamic register index
#pragma unroll
    for (int b = 0; b < R; b++)
        if (b == t) st = s_reg[b];
#pragma unroll
    for (int i = 0; i < NR; i++) {
        uint32_t o = s_thr;
        asm volatile("" : "+r"(o));   // recompute the slots: keeping all of them live would spill
#pragma unroll
        for (int b = 0; b < R; b++)
            if (i & (1 << b)) o ^= s_reg[b];
        const bool ctl = tctl && (cbit < 0 || ((i >> cbit) & 1));
        const C v = buf[ctl ? (o ^ st) : o];
        if (y) {
            if ((i >> t) & 1) { a[i].x = -v.y; a[i].y = v.x; }
            else { a[i].x = v.y; a[i].y = -v.x; }
        } else {
            a[i] = v;
        }
    }
}

// Run a phase's ops on the thread's amplitudes. ops/coefs: the op records
// and the coefficient array their coef indices refer to; (tpr, tpi): the
// per-thread phase of diagonal gates on thread bits; buf, s_thr, s_reg: the
// tile buffer and the thread's slot layout of this phase (permutations).
template <typename Real, int R>
__device__ __forceinline__ void run_ops(typename CT<Real>::T (&a)[1 << R], const Op *__restrict__ opsp, uint32_t count,
                                        const Real *__restrict__ coefs, int tid, Real &tpr, Real &tpi,
                                        typename CT<Real>::T *buf, uint32_t s_thr, const uint32_t (&s_reg)[R]) {
    constexpr int NR = 1 << R;
    for (uint32_t o = 0; o < count; o++) {
        const Op op = opsp[o];
        const Real *cf = coefs + op.coef;
        switch (op.kind) {
        case OP_X:
            perm_smem<NR, R>(a, buf, s_thr, s_reg, op.a, -1, true, false);
            break;
        case OP_Y:
            perm_smem<NR, R>(a, buf, s_thr, s_reg, op.a, -1, true, true);
            break;
        case OP_CX:
            perm_smem<NR, R>(a, buf, s_thr, s_reg, op.b, op.a, true, false);
            break;
        case OP_CXT:
            perm_smem<NR, R>(a, buf, s_thr, s_reg, op.b, -1, ((tid >> op.tb) & 1) != 0, false);
            break;
        case OP_H:
            with_bit<R>(op.a, [&](auto bc) { op_h<NR, decltype(bc)::value>(a); });
            break;
        case OP_U2:
            with_bit<R>(op.a, [&](auto bc) { op_u2<NR, decltype(bc)::value>(a, cf); });
            break;
        case OP_RX: {
            const Real c = cf[0], s = cf[1];
            with_bit<R>(op.a, [&](auto bc) { op_rx<NR, decltype(bc)::value>(a, c, s); });
        } break;
        case OP_RY: {
            const Real c = cf[0], s = cf[1];
            with_bit<R>(op.a, [&](auto bc) { op_ry<NR, decltype(bc)::value>(a, c, s); });
        } break;
        case OP_RXS: {
            const Real t = cf[0];
            if (op.b == 0) with_bit<R>(op.a, [&](auto bc) { op_rxs<NR, decltype(bc)::value, 0>(a, t); });
            else with_bit<R>(op.a, [&](auto bc) { op_rxs<NR, decltype(bc)::value, 1>(a, t); });
        } break;
        case OP_RYS: {
            const Real t = cf[0];
            if (op.b == 0) with_bit<R>(op.a, [&](auto bc) { op_rys<NR, decltype(bc)::value, 0>(a, t); });
            else with_bit<R>(op.a, [&](auto bc) { op_rys<NR, decltype(bc)::value, 1>(a, t); });
        } break;
        case OP_U2S: {
            const Real ur = cf[0], ui = cf[1], vr = cf[2], vi = cf[3], wr = cf[4], wi = cf[5];
            if (op.b == 0)
                with_bit<R>(op.a, [&](auto bc) { op_u2s<NR, decltype(bc)::value, 0>(a, ur, ui, vr, vi, wr, wi); });
            else
                with_bit<R>(op.a, [&](auto bc) { op_u2s<NR, decltype(bc)::value, 1>(a, ur, ui, vr, vi, wr, wi); });
        } break;
        case OP_D: {
            const Real d0r = cf[0], d0i = cf[1], d1r = cf[2], d1i = cf[3];
            with_bit<R>(op.a, [&](auto bc) { op_d<NR, decltype(bc)::value>(a, d0r, d0i, d1r, d1i); });
        } break;
        case OP_P: {
            const Real dr = cf[0], di = cf[1];
            with_bit<R>(op.a, [&](auto bc) { op_p<NR, decltype(bc)::value>(a, dr, di); });
        } break;
        case OP_Z:
            with_bit<R>(op.a, [&](auto bc) { op_z<NR, decltype(bc)::value>(a); });
            break;
        case OP_CP: {
            const Real dr = cf[0], di = cf[1];
            with_bit<R>(op.a, [&](auto ac) {
                with_bit<R>(op.b, [&](auto bc) {
                    constexpr int A = decltype(ac)::value, B = decltype(bc)::value;
                    if constexpr (A != B) op_cp<NR, A, B>(a, dr, di);
                });
            });
        } break;
        case OP_CZ:
            with_bit<R>(op.a, [&](auto ac) {
                with_bit<R>(op.b, [&](auto bc) {
                    constexpr int A = decltype(ac)::value, B = decltype(bc)::value;
                    if constexpr (A != B) op_cz<NR, A, B>(a);
                });
            });
            break;
        case OP_CPT:
            if ((tid >> op.tb) & 1) {
                const Real dr = cf[0], di = cf[1];
                with_bit<R>(op.a, [&](auto bc) { op_p<NR, decltype(bc)::value>(a, dr, di); });
            }
            break;
        case OP_CZT:
            if ((tid >> op.tb) & 1)
                with_bit<R>(op.a, [&](auto bc) { op_z<NR, decltype(bc)::value>(a); });
            break;
        case OP_TD: {
            const int bit = (tid >> op.tb) & 1;
            const Real dr = bit ? cf[2] : cf[0], di = bit ? cf[3] : cf[1];
            const Real x = tpr, y = tpi;
            tpr = x * dr - y * di;
            tpi = x * di + y * dr;
        } break;
        case OP_TP2:
            if (((tid >> op.tb) & 1) && ((tid >> op.b) & 1)) {
                const Real dr = cf[0], di = cf[1];
                const Real x = tpr, y = tpi;
                tpr = x * dr - y * di;
                tpi = x * di + y * dr;
            }
            break;
        case OP_DIAG:
#pragma unroll
            for (int i = 0; i < NR; i++) cmul_in(a[i], cf[2 * i], cf[2 * i + 1]);
            break;
        case OP_TAPPLY:
#pragma unroll
            for (int i = 0; i < NR; i++) cmul_in(a[i], tpr, tpi);
            tpr = Real(1);
            tpi = Real(0);
            break;
        default:
            break;
        }
    }
}

}  // namespace hisv
