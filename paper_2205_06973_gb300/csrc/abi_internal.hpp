// Internal definitions of the C-ABI handles, shared by abi.cpp and batch_abi.cpp.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hisvsim.h"
#include "jit.hpp"
#include "partition.hpp"
#include "planner.hpp"

using hisv::GateRef;
using hisv::Op;
using hisv::Phase;
using hisv::Program;

namespace hisv {

// Device allocations of the library are stream-ordered (the device memory
// pool): allocating or freeing never synchronises the whole device, so
// states and batches on other streams keep running.
inline cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st) { return cudaMallocAsync(p, bytes, st); }
inline void dev_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}
void set_last_error(const std::string &msg);
}

struct DevProgram {
    int dev = -1;
    Phase *d_phases = nullptr;
    Op *d_ops = nullptr;
    void *d_coefs = nullptr;
    uint8_t *d_aimg = nullptr;      // R images of the dense parts
    uint8_t *d_pimg = nullptr;      // R images of the dense pairs (two per pass)
};

struct sv_state {
    int n = 0;
    sv_precision prec = SV_C64;
    void *buf = nullptr;
    size_t bytes = 0;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int tile = 0;
    int dev = 0;
    double *d_partials = nullptr;   // kProbBlocks + 1 doubles; the last holds the norm
    double h_norm = 0.0;            // norm read back from the device
    int *d_err = nullptr;           // device error word of bounded waits (0 = none)
    double *d_dnorm = nullptr;      // norm accumulators of one apply's dense passes
    size_t dnorm_cap = 0;           // (1 + tensor-core passes), grown on demand
    void *d_stage = nullptr;        // double2 staging of double-float downloads (allocated on first use)
};

struct sv_plan {
    int n = 0;
    sv_method method = SV_PART_NONE;
    int k = 0;
    std::vector<GateRef> gates;
    std::vector<uint32_t> pog;
    uint32_t n_parts = 0;
    int max_part = 0;                                                      // qubits of the largest part
    std::vector<uint32_t> inner;        // second-level part of each gate (multi-level plans), else empty
    uint32_t n_inner = 0;
    int k2 = 0;
    std::map<std::tuple<bool, int, int>, std::unique_ptr<Program>> host_progs;   // (fp64, t, dense)
    std::map<std::tuple<int, bool, int, int>, DevProgram> dev_progs;             // (dev, fp64, t, dense)
    std::vector<std::vector<double>> mats;                                 // gatewise matrices
    std::map<std::tuple<int, int, int>, std::unique_ptr<hisv::JitProgram>> jit_progs;   // (precision, t, dense)
    // the caches above are filled on first use; several host threads may
    // apply one plan (map nodes never move, so returned pointers stay valid)
    std::recursive_mutex mu;
};

