// Batched persistent kernel: thousands of small, uneven circuits in one launch.
//
// Every circuit's plan is compiled for 2^9-amplitude tiles (32 lanes x 16
// amplitudes), so one warp executes one tile of one part with warp-private
// shared memory and no CTA-wide barrier. A device work list holds items
// (circuit, part, range of tiles) in wave order: the first parts of all
// circuits, then the second parts, and so on. Warps take items with an
// atomic ticket; an item of part w of circuit c starts once the circuit's
// tile counter shows that all tiles of its parts 0..w-1 are done (a bounded
// acquire spin), and bumps the counter with release semantics when it ends.
// An item only waits on items with smaller tickets, which running warps
// already hold, so the queue cannot deadlock.
#include <cuda_runtime.h>

#include <cstdint>

#include "batch.hpp"
#include "ops.cuh"

namespace hisv {

namespace {

constexpr int BT = BATCH_TILE_QUBITS;   // tile qubits
constexpr int BR = BATCH_REG_BITS;      // register bits per lane
constexpr int BNR = 1 << BR;
constexpr uint32_t BATCH_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t deposit_b(uint64_t v, uint64_t mask) {
    uint64_t out = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (v & 1) out |= low;
        v >>= 1;
        mask ^= low;
    }
    return out;
}

}  // namespace

__global__ void __launch_bounds__(256) k_batch(float2 *__restrict__ svbase, const BatchItem *__restrict__ items,
                                              uint32_t n_items, const uint64_t *__restrict__ circ_off,
                                              const PartLaunch *__restrict__ parts, const Phase *__restrict__ phases,
                                              const Op *__restrict__ ops, const float *__restrict__ coefs,
                                              uint32_t *__restrict__ done, uint32_t *__restrict__ head,
                                              int *__restrict__ err) {
    extern __shared__ __align__(16) float2 bsm[];
    const int lane = threadIdx.x & 31;
    float2 *const wsm = bsm + (threadIdx.x >> 5) * (1 << BT);
    float2 a[BNR];
    while (true) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(head, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const BatchItem I = items[it];
        if (I.wait) {
            int ok = 1;
            if (lane == 0) {
                uint32_t k = 0;
                while (ld_acquire(done + I.circuit) < I.wait) {
                    if (++k > BATCH_WAIT_LIMIT) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
        }
        const PartLaunch &P = parts[I.part];
        float2 *const sv = svbase + circ_off[I.circuit];
        // copy layout: tile element = lane (slots 0..4) | i << 5 (slots 5..9)
        uint64_t c_thr = 0;
        uint32_t s_cthr = 0;
#pragma unroll
        for (int j = 0; j < BT - BR; j++)
            if ((lane >> j) & 1) {
                c_thr |= 1ull << P.tile_q[j];
                s_cthr ^= swz<float>(j);
            }
        for (uint32_t tile = I.tile_begin; tile < I.tile_begin + I.tile_count; tile++) {
            const uint64_t base = deposit_b(tile, P.outer_mask) | c_thr;
#pragma unroll
            for (int i = 0; i < BNR; i++) {
                uint64_t go = 0;
                uint32_t so = s_cthr;
#pragma unroll
                for (int b = 0; b < BR; b++)
                    if (i & (1 << b)) {
                        go |= 1ull << P.tile_q[BT - BR + b];
                        so ^= swz<float>(BT - BR + b);
                    }
                wsm[so] = __ldcg(sv + (base | go));
            }
            __syncwarp();
            float tpr = 1.0f, tpi = 0.0f;
            uint32_t s_thr = 0, s_reg[BR];
            for (uint32_t p = 0; p < P.n_phases; p++) {
                const Phase ph = phases[P.phase_begin + p];
                if (p > 0) {   // transpose through the warp's shared tile
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < BNR; i++) {
                        uint32_t o = s_thr;
#pragma unroll
                        for (int b = 0; b < BR; b++)
                            if (i & (1 << b)) o ^= s_reg[b];
                        wsm[o] = a[i];
                    }
                    __syncwarp();
                }
                s_thr = 0;
#pragma unroll
                for (int j = 0; j < BT - BR; j++)
                    if ((lane >> j) & 1) s_thr ^= swz<float>(ph.thr[j]);
#pragma unroll
                for (int b = 0; b < BR; b++) s_reg[b] = swz<float>(ph.reg[b]);
#pragma unroll
                for (int i = 0; i < BNR; i++) {
                    uint32_t o = s_thr;
#pragma unroll
                    for (int b = 0; b < BR; b++)
                        if (i & (1 << b)) o ^= s_reg[b];
                    a[i] = wsm[o];
                }
                run_ops<float, BR>(a, ops + ph.op_begin, ph.op_count, coefs, lane, tpr, tpi, wsm, s_thr, s_reg);
            }
            if (P.flags & PL_STORE_FACTOR) {
                const float gr = (float)P.gr, gi = (float)P.gi;
                const float fr = gr * tpr - gi * tpi, fi = gr * tpi + gi * tpr;
#pragma unroll
                for (int i = 0; i < BNR; i++) cmul_in(a[i], fr, fi);
            }
            {
                uint64_t toff = deposit_b(tile, P.outer_mask);
#pragma unroll
                for (int j = 0; j < BT - BR; j++)
                    if ((lane >> j) & 1) toff |= 1ull << P.store_thr_q[j];
#pragma unroll
                for (int i = 0; i < BNR; i++) {
                    uint64_t off = toff;
#pragma unroll
                    for (int b = 0; b < BR; b++)
                        if (i & (1 << b)) off |= 1ull << P.store_reg_q[b];
                    __stcg(sv + off, a[i]);
                }
            }
            __syncwarp();   // the warp's shared tile is reused by the next tile
        }
        if (lane == 0) {
            __threadfence();
            red_release_add(done + I.circuit, I.tile_count);
        }
        __syncwarp();
    }
}

// p[i] = |a_i|^2 over the concatenated states; one block per circuit also
// sums its norm in FP64.
__global__ void __launch_bounds__(256) k_batch_probs(const float2 *__restrict__ svbase,
                                                     const uint64_t *__restrict__ circ_off,
                                                     const uint32_t *__restrict__ circ_n, float *__restrict__ out,
                                                     double *__restrict__ norms) {
    __shared__ double red[8];
    const uint32_t c = blockIdx.x;
    const uint64_t off = circ_off[c], N = 1ull << circ_n[c];
    double acc = 0.0;
    for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const float2 v = __ldcs(svbase + off + i);
        const double p = (double)v.x * v.x + (double)v.y * v.y;
        if (out) out[off + i] = (float)p;
        acc += p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; w++) s += red[w];
        norms[c] = s;
    }
}

__global__ void k_batch_reset(float2 *__restrict__ svbase, const uint64_t *__restrict__ circ_off,
                              uint32_t n_circ, uint64_t total) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x)
        svbase[i] = make_float2(0.f, 0.f);
}

__global__ void k_batch_basis(float2 *__restrict__ svbase, const uint64_t *__restrict__ circ_off, uint32_t n_circ) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_circ) svbase[circ_off[c]] = make_float2(1.f, 0.f);
}

cudaError_t batch_prepare(int warps_per_cta, int *n_ctas) {
    const size_t smem = (size_t)warps_per_cta * (1u << BT) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 8192);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, warps_per_cta * 32, smem)) != cudaSuccess)
        return e;
    *n_ctas = sms * (per_sm < 1 ? 1 : per_sm);
    return cudaSuccess;
}

cudaError_t launch_batch(const BatchLaunch &B, int warps_per_cta, int n_ctas, cudaStream_t st) {
    const size_t smem = (size_t)warps_per_cta * (1u << BT) * sizeof(float2);
    k_batch<<<n_ctas, warps_per_cta * 32, smem, st>>>(B.svbase, B.items, B.n_items, B.circ_off, B.parts, B.phases,
                                                      B.ops, B.coefs, B.done, B.head, B.err);
    return cudaGetLastError();
}

cudaError_t launch_batch_probs(float2 *svbase, const uint64_t *circ_off, const uint32_t *circ_n, uint32_t n_circ,
                               float *out, double *norms, cudaStream_t st) {
    k_batch_probs<<<n_circ, 256, 0, st>>>(svbase, circ_off, circ_n, out, norms);
    return cudaGetLastError();
}

cudaError_t launch_batch_reset(float2 *svbase, const uint64_t *circ_off, uint32_t n_circ, uint64_t total,
                               cudaStream_t st) {
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_batch_reset<<<(unsigned)blocks, 256, 0, st>>>(svbase, circ_off, n_circ, total);
    k_batch_basis<<<(n_circ + 255) / 256, 256, 0, st>>>(svbase, circ_off, n_circ);
    return cudaGetLastError();
}

}  // namespace hisv
