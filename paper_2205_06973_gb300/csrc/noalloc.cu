// Allocation-free variant of the probability / norm reduction.
//
// sv_measure_probs uses FP64 block partial sums in a scratch buffer that
// sv_create allocates. sv_probs_noalloc takes the state by device pointer and
// keeps its partial sums in the file-scope device array below instead, so it
// makes no device allocation at all. The array (SV_NOALLOC_MAX_BLOCKS + 1
// doubles) is part of the loaded library image: every GPU that loads the
// library holds it until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/hisvsim.h"
#include "kernels.hpp"

namespace {

// partial sums of one call, then (last slot) the norm when the caller passes
// no norm output
static __device__ __align__(256) double g_probs_scratch[SV_NOALLOC_MAX_BLOCKS + 1];

// Device address of g_probs_scratch, looked up once per device with that
// device current (the host-side name of the array is not a device address).
std::mutex g_mu;
void *g_addr[64];
bool g_ready[64];

}  // namespace

namespace hisv {
void set_last_error(const std::string &msg);   // the message sv_last_error() returns
}

static sv_status noalloc_fail(sv_status st, const std::string &msg) {
    hisv::set_last_error(msg);
    return st;
}

extern "C" sv_status sv_probs_noalloc(const void *dev_state, int n_qubits, sv_precision prec, void *dev_probs,
                                      int out_fp64, double *dev_norm, int n_blocks, void *stream) {
    if (!dev_state) {
        return noalloc_fail(SV_ERR_ARG, "dev_state is NULL");
    }
    if (n_qubits < 1 || n_qubits > 36) {
        return noalloc_fail(SV_ERR_ARG, "n_qubits must be in [1, 36]");
    }
    if (prec != SV_C64 && prec != SV_C128 && prec != SV_C128DF) {
        return noalloc_fail(SV_ERR_ARG, "bad precision");
    }
    if (n_blocks == 0) n_blocks = SV_NOALLOC_DEFAULT_BLOCKS;
    if (n_blocks < 1 || n_blocks > SV_NOALLOC_MAX_BLOCKS) {
        return noalloc_fail(SV_ERR_ARG, "n_blocks must be in [1, " + std::to_string(SV_NOALLOC_MAX_BLOCKS) +
                        "]: the static scratch holds that many FP64 partial sums");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        return noalloc_fail(SV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= 64) {
        return noalloc_fail(SV_ERR_ARG, "device ordinal " + std::to_string(dev) +
                                            " is outside the 64 devices this entry point tracks");
    }
    // The address is looked up again on every call made outside a stream
    // capture (cheap, no allocation), so a device reset or a new context on
    // the same ordinal never leaves a stale pointer behind; during a capture
    // (where the lookup is not allowed) the last address found is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cap);
    if (e != cudaSuccess) {
        return noalloc_fail(SV_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            e = cudaGetSymbolAddress(&g_addr[dev], g_probs_scratch);
            if (e != cudaSuccess) {
                g_ready[dev] = false;
                return noalloc_fail(SV_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_ready[dev] = true;
        } else if (!g_ready[dev]) {
            return noalloc_fail(SV_ERR_ARG, "first call on this device made during a stream capture: call it "
                                            "once outside the capture first");
        }
        scratch = g_addr[dev];
    }
    double *partials = static_cast<double *>(scratch);
    double *norm = dev_norm ? dev_norm : partials + SV_NOALLOC_MAX_BLOCKS;
    e = hisv::launch_probs(prec != SV_C64, dev_state, n_qubits, dev_probs, out_fp64, partials, n_blocks, norm,
                           reinterpret_cast<cudaStream_t>(stream), prec == SV_C128DF);
    if (e != cudaSuccess) {
        return noalloc_fail(SV_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    return SV_OK;
}
