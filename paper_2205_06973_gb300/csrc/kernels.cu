// sm_103a kernels of the hierarchical state-vector simulator.
//
//  k_part  : one HBM pass of one part (Algorithm 1, Gather-Execute-Scatter).
//            Persistent CTAs gather the 2^t amplitudes of one outer
//            assignment with cp.async into shared memory (the next tile's
//            copy overlaps the current tile's compute), run the part's
//            register phases (2^R amplitudes per thread), transposing the
//            tile through XOR-swizzled shared memory between phases, and
//            scatter it back from registers.
//  k_gate1 / k_gate2 : the plain per-gate pass of Sec. III-A (comparator).
//  k_probs / k_sum   : |a_x|^2 and the norm with FP64 accumulation.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "kernels.hpp"
#include "ops.cuh"

namespace hisv {

// ------------------------------------------------------------------------
// part kernel
// ------------------------------------------------------------------------
// Asynchronous global -> shared copies (sm_80+ cp.async); 8-byte elements use
// the L1-allocating form, 16-byte elements the L2-only form.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Deposit the bits of v, lowest first, into the set bits of mask.
__device__ __forceinline__ uint64_t deposit64(uint64_t v, uint64_t mask) {
    uint64_t out = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (v & 1) out |= low;
        v >>= 1;
        mask ^= low;
    }
    return out;
}

// Minimum resident CTAs for the launch bound: two tile buffers of 2^T
// amplitudes in shared memory and about 168 registers per thread.
template <typename Real, int T, int R>
struct PartCfg {
    static constexpr int NT = 1 << (T - R);
    static constexpr int SMEM = 2 * (1 << T) * 2 * (int)sizeof(Real);
    static constexpr int BY_REG = 65536 / (168 * NT);
    static constexpr int BY_SMEM = (227 * 1024) / SMEM;
    static constexpr int MINB0 = BY_REG < BY_SMEM ? BY_REG : BY_SMEM;
    static constexpr int MINB = MINB0 < 1 ? 1 : MINB0;
};

// One part pass. Persistent CTAs walk the tiles (outer assignments) with a
// two-stage pipeline: while tile i is computed from registers, the
// cp.async copy of tile i+1 streams into the other shared buffer.
template <typename Real, int T, int R>
__global__ void __launch_bounds__(PartCfg<Real, T, R>::NT, PartCfg<Real, T, R>::MINB)
k_part(typename CT<Real>::T *__restrict__ sv, const __grid_constant__ PartLaunch L,
       const Phase *__restrict__ phases, const Op *__restrict__ ops, const Real *__restrict__ coefs,
       uint64_t n_tiles) {
    typedef typename CT<Real>::T C;
    constexpr int NR = 1 << R;
    constexpr int TB = T - R;
    constexpr int TILE = 1 << T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *const buf0 = reinterpret_cast<C *>(smem_raw);
    C *const buf1 = buf0 + TILE;
    const int tid = threadIdx.x;

    // copy layout: tile index = tid | (c << TB); thread bits on the lowest slots
    uint64_t c_thr = 0;
    uint32_t s_cthr = 0;
#pragma unroll
    for (int j = 0; j < TB; j++)
        if ((tid >> j) & 1) {
            c_thr |= 1ull << L.tile_q[j];
            s_cthr ^= swz<Real>(j);
        }
    uint64_t c_rs[R];
    uint32_t s_crs[R];
#pragma unroll
    for (int b = 0; b < R; b++) {
        c_rs[b] = 1ull << L.tile_q[TB + b];
        s_crs[b] = swz<Real>(TB + b);
    }
    auto issue = [&](uint64_t base, C *dst) {
        const C *src = sv + (base | c_thr);
#pragma unroll
        for (int i = 0; i < NR; i++) {
            uint64_t go = 0;
            uint32_t so = s_cthr;
#pragma unroll
            for (int b = 0; b < R; b++)
                if (i & (1 << b)) {
                    go |= c_rs[b];
                    so ^= s_crs[b];
                }
            cp_async<(int)sizeof(C)>(dst + so, src + go);
        }
    };

    C a[NR];
    uint64_t tile = blockIdx.x;
    uint64_t base = tile < n_tiles ? deposit64(tile, L.outer_mask) : 0;
    if (tile < n_tiles) issue(base, buf0);
    cp_async_commit();
    for (uint32_t it = 0; tile < n_tiles; tile += gridDim.x, it++) {
        C *const cur = (it & 1) ? buf1 : buf0;
        C *const nxt = (it & 1) ? buf0 : buf1;
        __syncthreads();   // every thread is done with nxt (it was cur two stages ago)
        const uint64_t ntile = tile + gridDim.x;
        const uint64_t nbase = ntile < n_tiles ? deposit64(ntile, L.outer_mask) : 0;
        if (ntile < n_tiles) issue(nbase, nxt);
        cp_async_commit();
        cp_async_wait<1>();  // this tile's copies have landed
        __syncthreads();

        Real tpr = Real(1), tpi = Real(0);   // per-thread phase of diagonal gates on thread bits
        uint32_t s_thr = 0, s_reg[R];
        for (uint32_t p = 0; p < L.n_phases; p++) {
            const Phase ph = phases[L.phase_begin + p];
            if (p > 0) {
                // transpose through shared memory: write with the previous layout
                __syncthreads();
#pragma unroll
                for (int i = 0; i < NR; i++) {
                    uint32_t o = s_thr;
#pragma unroll
                    for (int b = 0; b < R; b++)
                        if (i & (1 << b)) o ^= s_reg[b];
                    cur[o] = a[i];
                }
                __syncthreads();
            }
            s_thr = 0;
#pragma unroll
            for (int j = 0; j < TB; j++)
                if ((tid >> j) & 1) s_thr ^= swz<Real>(ph.thr[j]);
#pragma unroll
            for (int b = 0; b < R; b++) s_reg[b] = swz<Real>(ph.reg[b]);
#pragma unroll
            for (int i = 0; i < NR; i++) {
                uint32_t o = s_thr;
#pragma unroll
                for (int b = 0; b < R; b++)
                    if (i & (1 << b)) o ^= s_reg[b];
                a[i] = cur[o];
            }
            // Execute: the phase's gates
            run_ops<Real, R>(a, ops + ph.op_begin, ph.op_count, coefs, tid, tpr, tpi, cur, s_thr, s_reg);
        }
        // Scatter: the last phase's layout, with SWAP relabels applied; the
        // part factor and the last phase's per-thread phase are applied here
        if (L.flags & PL_STORE_FACTOR) {
            const Real gr = (Real)L.gr, gi = (Real)L.gi;
            const Real fr = gr * tpr - gi * tpi, fi = gr * tpi + gi * tpr;
#pragma unroll
            for (int i = 0; i < NR; i++) cmul_in(a[i], fr, fi);
        }
        {
            uint64_t toff = base;
#pragma unroll
            for (int j = 0; j < TB; j++)
                if ((tid >> j) & 1) toff |= 1ull << L.store_thr_q[j];
            uint64_t rs[R];
#pragma unroll
            for (int b = 0; b < R; b++) rs[b] = 1ull << L.store_reg_q[b];
#pragma unroll
            for (int i = 0; i < NR; i++) {
                uint64_t off = toff;
#pragma unroll
                for (int b = 0; b < R; b++)
                    if (i & (1 << b)) off |= rs[b];
                __stcs(sv + off, a[i]);
            }
        }
        base = nbase;
    }
    cp_async_wait<0>();
}

template <typename Real, int T>
static cudaError_t launch_part_t(void *sv, const PartLaunch &L, const Phase *phases, const Op *ops,
                                 const void *coefs, uint64_t n_tiles, cudaStream_t st) {
    constexpr int R = sizeof(Real) == 4 ? 5 : 4;
    typedef typename CT<Real>::T C;
    typedef PartCfg<Real, T, R> Cfg;
    auto kern = k_part<Real, T, R>;
    const size_t smem = 2 * (sizeof(C) << T);
    // per instantiation: devices on which the shared-memory limit was raised,
    // and the resident CTAs per SM found there
    // (set once under a lock; a thread that sees the device's bit sees its counts)
    static std::atomic<uint64_t> attr_set{0};
    static std::mutex mu;
    static int resident[64];
    static int sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!((attr_set.load(std::memory_order_acquire) >> dev) & 1)) {
        std::lock_guard<std::mutex> lk(mu);
        if (!((attr_set.load(std::memory_order_relaxed) >> dev) & 1)) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, Cfg::NT, smem);
            if (e != cudaSuccess) return e;
            e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            resident[dev] = nb < 1 ? 1 : nb;
            attr_set.fetch_or(1ull << dev, std::memory_order_release);
        }
    }
    uint64_t grid = (uint64_t)sms[dev] * resident[dev];
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, Cfg::NT, smem, st>>>(reinterpret_cast<C *>(sv), L, phases, ops,
                                                reinterpret_cast<const Real *>(coefs), n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_part(bool fp64, int t, void *sv, const PartLaunch &L, const Phase *phases,
                        const Op *ops, const void *coefs, uint64_t n_tiles, cudaStream_t st) {
    if (!fp64) {
        switch (t) {
        case 10: return launch_part_t<float, 10>(sv, L, phases, ops, coefs, n_tiles, st);
        case 11: return launch_part_t<float, 11>(sv, L, phases, ops, coefs, n_tiles, st);
        case 12: return launch_part_t<float, 12>(sv, L, phases, ops, coefs, n_tiles, st);
        case 13: return launch_part_t<float, 13>(sv, L, phases, ops, coefs, n_tiles, st);
        }
    } else {
        switch (t) {
        case 10: return launch_part_t<double, 10>(sv, L, phases, ops, coefs, n_tiles, st);
        case 11: return launch_part_t<double, 11>(sv, L, phases, ops, coefs, n_tiles, st);
        case 12: return launch_part_t<double, 12>(sv, L, phases, ops, coefs, n_tiles, st);
        }
    }
    return cudaErrorInvalidValue;
}


// ------------------------------------------------------------------------
// plain per-gate kernels
// ------------------------------------------------------------------------
template <typename Real> struct M2 { Real m[8]; };
template <typename Real> struct M4 { Real m[32]; };

template <typename Real>
__global__ void __launch_bounds__(256) k_gate1(typename CT<Real>::T *__restrict__ sv, int q, uint64_t npairs,
                                                const __grid_constant__ M2<Real> g) {
    typedef typename CT<Real>::T C;
    const uint64_t lomask = (1ull << q) - 1;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x0 = ((p & ~lomask) << 1) | (p & lomask);
        const uint64_t x1 = x0 | (1ull << q);
        const C x = sv[x0], y = sv[x1];
        C u, v;
        u.x = g.m[0] * x.x - g.m[1] * x.y + g.m[2] * y.x - g.m[3] * y.y;
        u.y = g.m[0] * x.y + g.m[1] * x.x + g.m[2] * y.y + g.m[3] * y.x;
        v.x = g.m[4] * x.x - g.m[5] * x.y + g.m[6] * y.x - g.m[7] * y.y;
        v.y = g.m[4] * x.y + g.m[5] * x.x + g.m[6] * y.y + g.m[7] * y.x;
        sv[x0] = u;
        sv[x1] = v;
    }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_gate2(typename CT<Real>::T *__restrict__ sv, int q0, int q1,
                                                uint64_t nquads, const __grid_constant__ M4<Real> g) {
    typedef typename CT<Real>::T C;
    const int lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const uint64_t m_lo = (1ull << lo) - 1, m_hi = (1ull << hi) - 1;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nquads;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = ((p & ~m_lo) << 1) | (p & m_lo);   // insert a zero bit at lo
        x = ((x & ~m_hi) << 1) | (x & m_hi);              // then at hi
        uint64_t idx[4];
        idx[0] = x;
        idx[1] = x | (1ull << q0);
        idx[2] = x | (1ull << q1);
        idx[3] = x | (1ull << q0) | (1ull << q1);
        C in[4];
#pragma unroll
        for (int l = 0; l < 4; l++) in[l] = sv[idx[l]];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            Real re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const Real mr = g.m[2 * (4 * r + c)], mi = g.m[2 * (4 * r + c) + 1];
                re += mr * in[c].x - mi * in[c].y;
                im += mr * in[c].y + mi * in[c].x;
            }
            C o;
            o.x = re;
            o.y = im;
            sv[idx[r]] = o;
        }
    }
}

static unsigned grid_for(uint64_t work, int threads) {
    uint64_t b = (work + threads - 1) / threads;
    const uint64_t cap = 152ull * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_gate1(bool fp64, void *sv, int n, int q, const double *m, cudaStream_t st) {
    const uint64_t np = 1ull << (n - 1);
    if (!fp64) {
        M2<float> g;
        for (int i = 0; i < 8; i++) g.m[i] = (float)m[i];
        k_gate1<float><<<grid_for(np, 256), 256, 0, st>>>((float2 *)sv, q, np, g);
    } else {
        M2<double> g;
        for (int i = 0; i < 8; i++) g.m[i] = m[i];
        k_gate1<double><<<grid_for(np, 256), 256, 0, st>>>((double2 *)sv, q, np, g);
    }
    return cudaGetLastError();
}

cudaError_t launch_gate2(bool fp64, void *sv, int n, int q0, int q1, const double *m, cudaStream_t st) {
    const uint64_t nq = 1ull << (n - 2);
    if (!fp64) {
        M4<float> g;
        for (int i = 0; i < 32; i++) g.m[i] = (float)m[i];
        k_gate2<float><<<grid_for(nq, 256), 256, 0, st>>>((float2 *)sv, q0, q1, nq, g);
    } else {
        M4<double> g;
        for (int i = 0; i < 32; i++) g.m[i] = m[i];
        k_gate2<double><<<grid_for(nq, 256), 256, 0, st>>>((double2 *)sv, q0, q1, nq, g);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// probabilities and norm
// ------------------------------------------------------------------------
// Real and imaginary part of a stored amplitude, in FP64: complex64
// (float2), complex128 (double2) or double-float complex128 (float4: re.hi,
// re.lo, im.hi, im.lo; each part is the sum of its two floats).
__device__ __forceinline__ void amp_parts(const float2 &v, double &re, double &im) {
    re = (double)v.x;
    im = (double)v.y;
}
__device__ __forceinline__ void amp_parts(const double2 &v, double &re, double &im) {
    re = v.x;
    im = v.y;
}
__device__ __forceinline__ void amp_parts(const float4 &v, double &re, double &im) {
    re = (double)v.x + (double)v.y;
    im = (double)v.z + (double)v.w;
}

template <typename E, typename Out>
__global__ void __launch_bounds__(256) k_probs(const E *__restrict__ sv, uint64_t N,
                                                Out *__restrict__ out, double *__restrict__ partials) {
    __shared__ double red[8];
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const E v = __ldcs(sv + i);
        double re, im;
        amp_parts(v, re, im);
        const double p = re * re + im * im;
        if (out) out[i] = (Out)p;
        acc += p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_sum(const double *__restrict__ partials, int nb, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_probs(bool fp64, const void *sv, int n, void *out, int out_fp64, double *partials,
                         int nblocks, double *d_norm, cudaStream_t st, bool df) {
    const uint64_t N = 1ull << n;
    uint64_t need = (N + 255) / 256;
    int nb = (int)(need < (uint64_t)nblocks ? need : (uint64_t)nblocks);
    if (nb < 1) nb = 1;
    if (df) {
        if (out_fp64) k_probs<float4, double><<<nb, 256, 0, st>>>((const float4 *)sv, N, (double *)out, partials);
        else k_probs<float4, float><<<nb, 256, 0, st>>>((const float4 *)sv, N, (float *)out, partials);
    } else if (!fp64) {
        if (out_fp64) k_probs<float2, double><<<nb, 256, 0, st>>>((const float2 *)sv, N, (double *)out, partials);
        else k_probs<float2, float><<<nb, 256, 0, st>>>((const float2 *)sv, N, (float *)out, partials);
    } else {
        if (out_fp64) k_probs<double2, double><<<nb, 256, 0, st>>>((const double2 *)sv, N, (double *)out, partials);
        else k_probs<double2, float><<<nb, 256, 0, st>>>((const double2 *)sv, N, (float *)out, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum<<<1, 256, 0, st>>>(partials, nb, d_norm);
    return cudaGetLastError();
}

// Summary of the probability distribution without writing it: per block the
// FP64 sum of |a_x|^2 and the largest |a_x|^2 with its index (ties to the
// smaller index), then one block combines them.
__device__ __forceinline__ void better(double &p, uint64_t &i, double q, uint64_t j) {
    if (q > p || (q == p && j < i)) {
        p = q;
        i = j;
    }
}

template <typename E>
__global__ void __launch_bounds__(256) k_summary(const E *__restrict__ sv, uint64_t N,
                                                  double *__restrict__ sums, double *__restrict__ maxs,
                                                  uint64_t *__restrict__ idxs) {
    __shared__ double rs[8], rm[8];
    __shared__ uint64_t ri[8];
    double acc = 0.0, best = -1.0;
    uint64_t bi = ~0ull;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const E v = __ldcs(sv + i);
        double re, im;
        amp_parts(v, re, im);
        const double p = re * re + im * im;
        acc += p;
        better(best, bi, p, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double q = __shfl_xor_sync(0xffffffffu, best, o);
        const uint64_t j = __shfl_xor_sync(0xffffffffu, bi, o);
        better(best, bi, q, j);
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = acc;
        rm[threadIdx.x >> 5] = best;
        ri[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, m = -1.0;
        uint64_t mi = ~0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            s += rs[w];
            better(m, mi, rm[w], ri[w]);
        }
        sums[blockIdx.x] = s;
        maxs[blockIdx.x] = m;
        idxs[blockIdx.x] = mi;
    }
}

// out[0] = sum |a|^2, out[1] = |a_0|^2, out[2] = max |a_x|^2, out[3] = its index (bits)
template <typename E>
__global__ void k_summary_final(const E *__restrict__ sv, const double *__restrict__ sums,
                                const double *__restrict__ maxs, const uint64_t *__restrict__ idxs, int nb,
                                double *__restrict__ out) {
    __shared__ double rs[256], rm[256];
    __shared__ uint64_t ri[256];
    double s = 0.0, m = -1.0;
    uint64_t mi = ~0ull;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s += sums[i];
        better(m, mi, maxs[i], idxs[i]);
    }
    rs[threadIdx.x] = s;
    rm[threadIdx.x] = m;
    ri[threadIdx.x] = mi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            rs[threadIdx.x] += rs[threadIdx.x + w];
            better(rm[threadIdx.x], ri[threadIdx.x], rm[threadIdx.x + w], ri[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double re, im;
        amp_parts(sv[0], re, im);
        out[0] = rs[0];
        out[1] = re * re + im * im;
        out[2] = rm[0];
        out[3] = __longlong_as_double((long long)ri[0]);
    }
}

cudaError_t launch_summary(bool fp64, const void *sv, int n, double *scratch, int nblocks, double *out,
                           cudaStream_t st, bool df) {
    const uint64_t N = 1ull << n;
    uint64_t need = (N + 255) / 256;
    int nb = (int)(need < (uint64_t)nblocks ? need : (uint64_t)nblocks);
    if (nb < 1) nb = 1;
    double *sums = scratch, *maxs = scratch + nblocks;
    uint64_t *idxs = reinterpret_cast<uint64_t *>(scratch + 2 * nblocks);
    if (df) {
        k_summary<float4><<<nb, 256, 0, st>>>((const float4 *)sv, N, sums, maxs, idxs);
        k_summary_final<float4><<<1, 256, 0, st>>>((const float4 *)sv, sums, maxs, idxs, nb, out);
    } else if (fp64) {
        k_summary<double2><<<nb, 256, 0, st>>>((const double2 *)sv, N, sums, maxs, idxs);
        k_summary_final<double2><<<1, 256, 0, st>>>((const double2 *)sv, sums, maxs, idxs, nb, out);
    } else {
        k_summary<float2><<<nb, 256, 0, st>>>((const float2 *)sv, N, sums, maxs, idxs);
        k_summary_final<float2><<<1, 256, 0, st>>>((const float2 *)sv, sums, maxs, idxs, nb, out);
    }
    return cudaGetLastError();
}

// ALU peak probe: 8 independent FMA chains per thread (enough to cover the
// FMA latency), over a grid that fills every SM; the result is stored so the
// chains are not removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *__restrict__ out, int iters, T b, T c) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = (T)(threadIdx.x + j);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fma(x[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t alu_probe(bool fp64, double *flops_per_s, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256;
    void *out = nullptr;
    e = cudaMallocAsync(&out, (size_t)blocks * threads * 8, st);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    int iters = 256;
    for (int rep = 0; rep < 8 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, st);
        if (fp64) k_fma_probe<double><<<blocks, threads, 0, st>>>((double *)out, iters, 0.999999, 1e-7);
        else k_fma_probe<float><<<blocks, threads, 0, st>>>((float *)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
        if (ms > 0.f) best = flops / (ms * 1e-3) > best ? flops / (ms * 1e-3) : best;
        if (ms < 20.f && iters < (1 << 24)) iters *= 4;   // grow to a launch of tens of milliseconds
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (e != cudaSuccess) return e;
    *flops_per_s = best;
    return cudaGetLastError();
}

template <typename Real>
__global__ void k_set_one(typename CT<Real>::T *sv, uint64_t idx) {
    typename CT<Real>::T v;
    v.x = Real(1);
    v.y = Real(0);
    sv[idx] = v;
}

__global__ void k_set_one_df(float4 *sv, uint64_t idx) { sv[idx] = make_float4(1.f, 0.f, 0.f, 0.f); }

cudaError_t launch_set_basis(bool fp64, void *sv, int n, uint64_t idx, cudaStream_t st, bool df) {
    const size_t bytes = (fp64 || df ? 16ull : 8ull) << n;
    cudaError_t e = cudaMemsetAsync(sv, 0, bytes, st);
    if (e != cudaSuccess) return e;
    if (df) k_set_one_df<<<1, 1, 0, st>>>((float4 *)sv, idx);
    else if (fp64) k_set_one<double><<<1, 1, 0, st>>>((double2 *)sv, idx);
    else k_set_one<float><<<1, 1, 0, st>>>((float2 *)sv, idx);
    return cudaGetLastError();
}

// Double-float representation (Dekker 1971): a double d is held as the
// unevaluated sum hi + lo of two floats, hi = d rounded to float and lo =
// (d - hi) rounded to float (d - hi is exact in FP64). In place: each element
// is read before it is written.
__global__ void __launch_bounds__(256) k_to_df(double2 *__restrict__ sv, uint64_t N) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const double2 v = sv[i];
        const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
        const float rl = __double2float_rn(v.x - (double)rh), il = __double2float_rn(v.y - (double)ih);
        reinterpret_cast<float4 *>(sv)[i] = make_float4(rh, rl, ih, il);
    }
}

// hi + lo back to FP64 (exact: lo lies below hi's last bit, the sum fits 53 bits).
__global__ void __launch_bounds__(256) k_from_df(const float4 *__restrict__ src, double2 *__restrict__ dst,
                                                 uint64_t N) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 v = src[i];
        dst[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

cudaError_t launch_to_df(void *sv, uint64_t n_amps, cudaStream_t st) {
    k_to_df<<<grid_for(n_amps, 256), 256, 0, st>>>((double2 *)sv, n_amps);
    return cudaGetLastError();
}

cudaError_t launch_from_df(const void *src, void *dst, uint64_t n_amps, cudaStream_t st) {
    k_from_df<<<grid_for(n_amps, 256), 256, 0, st>>>((const float4 *)src, (double2 *)dst, n_amps);
    return cudaGetLastError();
}

}  // namespace hisv
