// Dense fused-part kernel on the sm_103a tensor cores (tcgen05 + TMEM).
//
// A part on 6 qubits is the 64x64 complex matrix U (the product of its
// gates). With amplitudes stored as interleaved (re, im) floats, the part
// maps every column x (64 amplitudes that share the other n - 6 bits) to
// R x, R the 128x128 real block form R[2i+c][2j+d] of U. A CTA tile is 128
// columns (the lowest 7 non-part qubits); with the tile as the MMA's A
// operand and R as its B operand the GEMM is
//     D[128 x 128] = X^T[128 x 128] . R^T      (M = 128 columns, N = 128, K = 128)
// so D row n (TMEM lane n) holds the 64 output amplitudes of column n. It
// runs as split BF16: R = R_hi + R_lo, X = X_hi + X_lo and
// D = X_hi R_hi + X_lo R_hi + X_hi R_lo with FP32 accumulation in tensor
// memory (the dropped X_lo R_lo term is below 2^-16 relative).
//
// Data path: HBM -> registers -> tensor memory -> registers -> HBM. Only the
// 64 KiB image of R (resident for the whole launch) is read from shared
// memory, by the MMAs, so the tile crosses the SM's shared-memory datapath
// only as global loads and stores.
//
// Warp-specialised persistent CTA (13 warps, one CTA per SM):
//  * 8 converter warps (two per TMEM lane quarter): thread (lane n, half h)
//    loads amplitudes 32h..32h+31 of column n (for a fixed amplitude the
//    warp's 32 columns are consecutive in memory when the column qubits are
//    the lowest ones), splits them to BF16 hi/lo, and writes them with
//    tcgen05.st into the TMEM A buffer of the tile (two buffers). They warm
//    L2 with their next tile (one 128-byte line per lane; one tile ahead
//    measured 2-4 % faster than two, and more than three or four).
//  * one thread of the MMA warp issues the 24 MMAs (K = 16 each) of a tile
//    into one of two TMEM accumulators and commits them to the accumulator's
//    full barrier (which also frees the tile's A buffer);
//  * 4 epilogue warps (one per lane quarter) read the accumulator
//    (tcgen05.ld; lane n = column n, 16 amplitudes at a time), apply the
//    norm correction and store complete (re, im) amplitudes, coalesced like
//    the loads.
// TMEM: accumulators at columns 0 and 128, A buffers at 256 and 384 (hi in
// the first 64 columns, lo in the next 64): all 512 columns, so the launch
// asks for enough shared memory to keep a second CTA off the SM. Every
// mbarrier wait is bounded; on expiry the role records an error code and
// leaves its loop, the MMA thread waits (bounded) for its last commit, and
// the TMEM is freed on exit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "dense.hpp"
#include "dense_common.cuh"

namespace hisv {

using namespace dense_detail;

constexpr int EPI_WARPS = 4;      // one per TMEM lane quarter (warp w: quarter w)
constexpr int CONV_WARPS = 8;     // two per TMEM lane quarter (warp 4 + w: quarter w % 4, half w / 4)
constexpr int MMA_WARP = EPI_WARPS + CONV_WARPS;
constexpr int DENSE_THREADS = (MMA_WARP + 1) * 32;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr uint32_t TMEM_COLS = 512;                  // D0, D1, A0, A1 at 0, 128, 256, 384
// R image + barriers; sized above half of the SM's shared memory so that a
// second CTA (which would wait for the TMEM this one holds) cannot share the SM
constexpr uint32_t DENSE_SMEM = 120 * 1024;
constexpr uint32_t WAIT_LIMIT = 1u << 24;            // bounded mbarrier polls
static_assert(DENSE_A_BYTES + 1024 + 16 * CONV_THREADS + 1024 <= (int)DENSE_SMEM, "shared memory layout");

template <int W>
__global__ void __launch_bounds__(DENSE_THREADS, 1)
k_dense6(float2 *__restrict__ sv, const __grid_constant__ DenseLaunch L, const uint8_t *__restrict__ a_img,
         uint64_t n_tiles, int *__restrict__ err, double *__restrict__ dn, uint32_t dense_idx) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *const base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *const sR = base;                                               // R image (B operand)
    uint64_t *const bars = reinterpret_cast<uint64_t *>(base + DENSE_A_BYTES);
    uint64_t *const afull = bars, *const dfull = bars + 2, *const dempty = bars + 4;
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(base + DENSE_A_BYTES + 128);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < DENSE_A_BYTES / 16; i += DENSE_THREADS)
        reinterpret_cast<uint4 *>(sR)[i] = reinterpret_cast<const uint4 *>(a_img)[i];
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            mbar_init(&afull[b], CONV_THREADS);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], EPI_THREADS);
        }
        mbar_init_fence();
    }
    if (warp == MMA_WARP) {
        tmem_alloc(tslot, TMEM_COLS);
        tmem_relinquish();
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // R image visible to the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    // the previous kernel on the stream (another pass) has completed and its
    // writes (state, norm accumulators) are visible from here on
    asm volatile("griddepcontrol.wait;\n" ::: "memory");

    // per-thread geometry shared by converters and epilogue: TMEM lane
    // quarter q and amplitude half h of the warp; column n = 32 q + lane
    const int q = warp & 3, h = warp >= EPI_WARPS ? ((warp - EPI_WARPS) >> 2) & 1 : 0;
    const uint32_t n_col = 32 * q + lane;
    uint64_t coff = 0;                                   // column n's bits on the column qubits
#pragma unroll
    for (int b = 0; b < DENSE_COLS; b++)
        if ((n_col >> b) & 1) coff |= 1ull << L.col_q[b];
    uint64_t pbit[DENSE_K];
#pragma unroll
    for (int b = 0; b < DENSE_K; b++) pbit[b] = 1ull << L.part_q[b];
    const uint64_t hoff = h ? pbit[DENSE_K - 1] : 0ull;  // amplitude bit 5 = the half
    const uint64_t dgrid = deposit_bits(gridDim.x, L.outer_mask);

    if (warp >= EPI_WARPS && warp < MMA_WARP) {
        // ------------------------------------------------------ converters
        // L2 warm-up lines of a tile: qubits 0..3 are tile qubits, so a tile
        // is 512 lines of 128 bytes, line lam at the deposit of lam into the
        // tile's qubits above 3
        const int ctid = tid - EPI_THREADS;
        const uint64_t all = L.n >= 64 ? ~0ull : ((1ull << L.n) - 1);
        const uint64_t tile_q = all & ~L.outer_mask & ~0xFull;
        uint64_t *const lineoff = reinterpret_cast<uint64_t *>(base + DENSE_A_BYTES + 1024) + 2 * ctid;
#pragma unroll
        for (int u = 0; u < 2; u++) lineoff[u] = deposit_bits((uint64_t)(ctid + 256 * u), tile_q);
        double in_norm = 0.0;   // sum of |a|^2 of the input (first dense pass of an apply)
        uint64_t tb = deposit_bits(blockIdx.x, L.outer_mask);
        uint64_t tpf = masked_add(tb, dgrid, L.outer_mask);   // the CTA's next tile
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, i++) {
            const uint32_t b = i & 1;
            // the MMAs of tile i - 2 (same A buffer) have completed
            // warp-uniform: the tcgen05 stores below are .sync.aligned
            if (!__all_sync(0xffffffffu, i < 2 || mbar_wait(&dfull[b], ((i >> 1) - 1) & 1, WAIT_LIMIT))) {
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            if (tile + gridDim.x < n_tiles) {
#pragma unroll
                for (int u = 0; u < 2; u++) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(sv + (tpf | lineoff[u])));
            }
            const float2 *const src = sv + (tb | coff | hoff);
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + 256 + 128 * b + 32 * h;
            float tile_in = 0.0f;   // FP32 partial of this tile, folded into the FP64 sum
#pragma unroll
            for (int g = 0; g < 2; g++) {   // two rounds of 16 loads (the lines are in L2 by now)
                float2 x[16];
#pragma unroll
                for (int j = 0; j < 16; j += W) {
                    const int m = 16 * g + j;   // its low log2(W) bits are 0: W consecutive amplitudes
                    uint64_t o = 0;
#pragma unroll
                    for (int bb = 0; bb < 5; bb++)
                        if ((m >> bb) & 1) o |= pbit[bb];
                    ld_amps<W>(src + o, x + j);
                }
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const float2 v = x[j];
                    tile_in = fmaf(v.x, v.x, fmaf(v.y, v.y, tile_in));
                    const __nv_bfloat162 bh = __floats2bfloat162_rn(v.x, v.y);
                    const float2 hf = __bfloat1622float2(bh);
                    const __nv_bfloat162 bl = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
                    hi[j] = *reinterpret_cast<const uint32_t *>(&bh);
                    lo[j] = *reinterpret_cast<const uint32_t *>(&bl);
                }
                tmem_st16(ta + 16 * g, hi);
                tmem_st16(ta + 64 + 16 * g, lo);
            }
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(&afull[b]);
            if (dense_idx == 0) in_norm += (double)tile_in;
            tb = masked_add(tb, dgrid, L.outer_mask);
            tpf = masked_add(tpf, dgrid, L.outer_mask);
        }
        if (dense_idx == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) in_norm += __shfl_xor_sync(0xffffffffu, in_norm, o);
            if (lane == 0) atomicAdd(dn, in_norm);
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, 128);
            const uint32_t sb = smem_u32(sR);
            uint32_t i = 0;
            for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, i++) {
                const uint32_t b = i & 1, u = i >> 1;
                if (!mbar_wait(&afull[b], u & 1, WAIT_LIMIT) ||
                    (i >= 2 && !mbar_wait(&dempty[b], (u - 1) & 1, WAIT_LIMIT))) {
                    atomicExch(err, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + 128 * b, a = tmem + 256 + 128 * b;
                uint32_t acc = 0;
#pragma unroll
                for (int p = 0; p < 3; p++) {
                    // p = 0: X_hi R_hi, 1: X_lo R_hi, 2: X_hi R_lo
                    const uint32_t xsel = p == 1 ? 64u : 0u, rsel = p == 2 ? 1u : 0u;
#pragma unroll
                    for (int ks = 0; ks < 8; ks++) {
                        const uint32_t ra = sb + (rsel * 2 + (ks >> 2)) * 16384 + (ks & 3) * 32;
                        umma_bf16_ts(d, a + xsel + 8 * ks, sw128_desc(ra), idesc, acc);
                        acc = 1;
                    }
                }
                umma_commit(&dfull[b]);    // accumulator ready, A buffer consumed
            }
            // the MMAs of the last tile complete before the TMEM is freed
            if (i > 0 && !mbar_wait(&dfull[(i - 1) & 1], ((i - 1) >> 1) & 1, WAIT_LIMIT)) atomicExch(err, 1);
        }
    } else {
        // ------------------------------------------------------ epilogue
        // unitarity: rescale to the input norm N0 measured by the first dense
        // pass, correcting the drift measured on the previous dense pass
        float scale = 1.0f;
        if (dense_idx > 0) {
            const double n0 = dn[0], prev = dn[dense_idx];
            if (n0 > 0.0 && prev > 0.0) scale = (float)sqrt(n0 / prev);
        }
        double out_norm = 0.0;
        uint64_t tb = deposit_bits(blockIdx.x, L.outer_mask);
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, i++) {
            const uint32_t b = i & 1, u = i >> 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&dfull[b], u & 1, WAIT_LIMIT))) {   // warp-uniform (tcgen05.ld)
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t td = tmem + ((uint32_t)(32 * q) << 16) + 128 * b;
            float2 *const dst = sv + (tb | coff);
            float tile_out = 0.0f;
#pragma unroll
            for (int g = 0; g < 4; g++) {   // 16 amplitudes (32 columns) at a time
                uint32_t r[32];
                tmem_ld32(td + 32 * g, r);
                tmem_ld_wait();
                if (g == 3) {
                    tc_fence_before();
                    mbar_arrive(&dempty[b]);
                }
#pragma unroll
                for (int j = 0; j < 16; j += W) {
                    const int m = 16 * g + j;
                    uint64_t o = 0;
#pragma unroll
                    for (int bb = 0; bb < 6; bb++)
                        if ((m >> bb) & 1) o |= pbit[bb];
                    float2 y[W];
#pragma unroll
                    for (int w = 0; w < W; w++) {
                        y[w] = make_float2(__uint_as_float(r[2 * (j + w)]) * scale,
                                           __uint_as_float(r[2 * (j + w) + 1]) * scale);
                        tile_out = fmaf(y[w].x, y[w].x, fmaf(y[w].y, y[w].y, tile_out));
                    }
                    st_amps<W>(dst + o, y);
                }
            }
            out_norm += (double)tile_out;
            tb = masked_add(tb, dgrid, L.outer_mask);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) out_norm += __shfl_xor_sync(0xffffffffu, out_norm, o);
        if (lane == 0) atomicAdd(dn + 1 + dense_idx, out_norm);
    }
    // the CTA's work is done: once every CTA got here, the next pass on the
    // stream may launch and run its prologue on the SMs this one leaves
    // (programmatic dependent launch; it waits for this grid before it
    // touches the state). Signalling only now keeps the waiting CTAs of the
    // next pass from occupying SMs that other streams' kernels could use.
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host ---
static uint16_t bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);   // inf / nan
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float bf16_to_f(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
static uint32_t sw128_off_host(uint32_t r, uint32_t k) {
    return r * 128u + ((((k >> 3) ^ (r & 7u)) & 7u) << 4) + ((k & 7u) << 1);
}

void dense_a_image(const double *U, std::vector<uint8_t> &img) {
    img.assign(DENSE_A_BYTES, 0);
    for (int r = 0; r < 128; r++)
        for (int k = 0; k < 128; k++) {
            const int i = r >> 1, c = r & 1, j = k >> 1, d = k & 1;
            const double ur = U[2 * (64 * i + j)], ui = U[2 * (64 * i + j) + 1];
            const double R = (c == d) ? ur : (c == 0 ? -ui : ui);
            const uint16_t hi = bf16_rne((float)R);
            const uint16_t lo = bf16_rne((float)(R - (double)bf16_to_f(hi)));
            const uint32_t kb = (uint32_t)k >> 6, off = sw128_off_host((uint32_t)r, (uint32_t)k & 63u);
            std::memcpy(&img[(0 * 2 + kb) * 16384 + off], &hi, 2);
            std::memcpy(&img[(1 * 2 + kb) * 16384 + off], &lo, 2);
        }
}

cudaError_t launch_dense6(void *sv, const DenseLaunch &L, const void *a_img, uint64_t n_tiles, int *d_err,
                          double *d_norms, uint32_t dense_idx, cudaStream_t st) {
    // per device: shared-memory limit raised and SM count cached, once
    // (double-checked: a thread that sees the bit sees the count)
    static std::atomic<uint64_t> attr_set{0};
    static std::mutex mu;
    static int sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!((attr_set.load(std::memory_order_acquire) >> dev) & 1)) {
        std::lock_guard<std::mutex> lk(mu);
        if (!((attr_set.load(std::memory_order_relaxed) >> dev) & 1)) {
            e = cudaFuncSetAttribute(k_dense6<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DENSE_SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_dense6<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DENSE_SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_dense6<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DENSE_SMEM);
            if (e != cudaSuccess) return e;
            e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            attr_set.fetch_or(1ull << dev, std::memory_order_release);
        }
    }
    if (reinterpret_cast<uintptr_t>(sv) & 15) return cudaErrorMisalignedAddress;
    uint64_t grid = (uint64_t)sms[dev];
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;
    // amplitudes per lane access: the part qubits 0, 1, ... in a row make the
    // amplitudes of a column consecutive (qubit 0 a column qubit: the lanes are)
    int z = 0;
    while (z < DENSE_K && L.part_q[z] == z) z++;
    const bool a32 = (reinterpret_cast<uintptr_t>(sv) & 31) == 0;
    float2 *const p = reinterpret_cast<float2 *>(sv);
    const uint8_t *const a = reinterpret_cast<const uint8_t *>(a_img);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(DENSE_THREADS);
    cfg.dynamicSmemBytes = DENSE_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (z >= 2 && a32)
        e = cudaLaunchKernelEx(&cfg, k_dense6<4>, p, L, a, n_tiles, d_err, d_norms, dense_idx);
    else if (z >= 1)
        e = cudaLaunchKernelEx(&cfg, k_dense6<2>, p, L, a, n_tiles, d_err, d_norms, dense_idx);
    else
        e = cudaLaunchKernelEx(&cfg, k_dense6<1>, p, L, a, n_tiles, d_err, d_norms, dense_idx);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace hisv
