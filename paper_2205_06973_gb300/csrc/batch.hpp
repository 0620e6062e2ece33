// Batched persistent launch over many small circuits (device side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "program.hpp"

namespace hisv {

// One queue item: tiles [tile_begin, tile_begin + tile_count) of part `part`
// (index into the concatenated PartLaunch array) of circuit `circuit`; it may
// start once done[circuit] >= wait (tiles of the circuit's earlier parts).
struct BatchItem {
    uint32_t circuit;
    uint32_t part;
    uint32_t tile_begin;
    uint32_t tile_count;
    uint32_t wait;
};

struct BatchLaunch {
    float2 *svbase;              // concatenated complex64 states
    const BatchItem *items;
    uint32_t n_items;
    const uint64_t *circ_off;    // first amplitude of each circuit's state
    const PartLaunch *parts;     // all circuits' parts (tile of 2^9 amplitudes)
    const Phase *phases;
    const Op *ops;
    const float *coefs;
    uint32_t *done;              // per-circuit finished-tile counters (zeroed per run)
    uint32_t *head;              // queue ticket (zeroed per run)
    int *err;                    // bounded-wait failure flag
};

constexpr int BATCH_TILE_QUBITS = 9;   // one warp's tile: 32 lanes x 16 amplitudes
constexpr int BATCH_REG_BITS = 4;      // tile qubits held in registers (16 amplitudes per lane)
constexpr int BATCH_MIN_QUBITS = 10;

// Raise the shared-memory limit and return the persistent grid size (CTAs
// resident on all SMs) for a CTA of warps_per_cta warps.
cudaError_t batch_prepare(int warps_per_cta, int *n_ctas);
cudaError_t launch_batch(const BatchLaunch &B, int warps_per_cta, int n_ctas, cudaStream_t st);
cudaError_t launch_batch_probs(float2 *svbase, const uint64_t *circ_off, const uint32_t *circ_n, uint32_t n_circ,
                               float *out, double *norms, cudaStream_t st);
cudaError_t launch_batch_reset(float2 *svbase, const uint64_t *circ_off, uint32_t n_circ, uint64_t total,
                               cudaStream_t st);

}  // namespace hisv
