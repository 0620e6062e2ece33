// Host-side launchers of the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "program.hpp"

namespace hisv {

// Register bits per thread of the part kernel: 5 for complex64, 4 for complex128.
inline int part_R(bool fp64) { return fp64 ? 4 : 5; }
inline int part_tmin() { return 10; }
inline int part_tmax(bool fp64) { return fp64 ? 12 : 13; }

// One pass of a part over the whole state (Algorithm 1): n_tiles = 2^(n - t) CTAs.
cudaError_t launch_part(bool fp64, int t, void *sv, const PartLaunch &L, const Phase *phases,
                        const Op *ops, const void *coefs, uint64_t n_tiles, cudaStream_t st);

// Plain one-pass-per-gate kernels (Sec. III-A): m is the 2x2 (8 reals) or 4x4
// (32 reals, local index l = b_q0 + 2 b_q1) complex matrix, row-major (re, im).
cudaError_t launch_gate1(bool fp64, void *sv, int n, int q, const double *m, cudaStream_t st);
cudaError_t launch_gate2(bool fp64, void *sv, int n, int q0, int q1, const double *m, cudaStream_t st);

// p[x] = |a_x|^2 (float or double out, may be null) and FP64 block partial sums
// of the norm reduced into *d_norm. partials has nblocks doubles.
cudaError_t launch_probs(bool fp64, const void *sv, int n, void *out, int out_fp64, double *partials,
                         int nblocks, double *d_norm, cudaStream_t st, bool df = false);

// Norm, |a_0|^2 and the largest |a_x|^2 with its index (ties to the smaller
// index), FP64, without a probability vector: scratch holds 3 * nblocks
// doubles, out 4 (out[3] holds the index's bits).
cudaError_t launch_summary(bool fp64, const void *sv, int n, double *scratch, int nblocks, double *out,
                           cudaStream_t st, bool df = false);
// FMA throughput of the CUDA cores in FP64 (fp64) or FP32, in FLOP/s (best of
// a few timed launches over every SM; synchronises the stream).
cudaError_t alu_probe(bool fp64, double *flops_per_s, cudaStream_t st);
cudaError_t launch_set_basis(bool fp64, void *sv, int n, uint64_t idx, cudaStream_t st, bool df = false);
// Double-float complex128 (df = true above): each part of an amplitude is the
// sum hi + lo of two floats, stored (re.hi, re.lo, im.hi, im.lo).
// launch_to_df converts n_amps double2 amplitudes in place; launch_from_df
// writes the double2 values of n_amps double-float amplitudes to dst.
cudaError_t launch_to_df(void *sv, uint64_t n_amps, cudaStream_t st);
cudaError_t launch_from_df(const void *src, void *dst, uint64_t n_amps, cudaStream_t st);

}  // namespace hisv
