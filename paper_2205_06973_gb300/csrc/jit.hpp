// Part kernels specialised for one plan: CUDA source generated from the
// compiled program (tile layout, register phases, ops with their
// coefficients) and compiled at run time with NVRTC for sm_103a.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "planner.hpp"

namespace hisv {

struct JitProgram {
    bool fp64 = false;
    int t = 0, R = 0;
    int threads = 0;                      // per CTA: 2^(t - R)
    size_t smem = 0;                      // two tile buffers
    std::vector<cudaLibrary_t> libs;      // one per compiled chunk of parts
    std::vector<cudaKernel_t> kern;       // per gate-list part (Program::parts order)
    uint64_t attr_devices = 0;            // devices on which the shared-memory limit was raised
    int resident[64] = {};                // CTAs per SM found there
    int sms[64] = {};
    double compile_s = 0.0;
};

// CUDA source of gate-list part i of prog (one extern "C" kernel named
// hisv_part_<i>); df: the complex128 program in double-float arithmetic on
// double-float amplitudes (16 bytes each, like complex128).
std::string jit_part_source(const Program &prog, size_t i, bool df = false);

// Generate and compile every gate-list part of prog (chunks compiled in
// parallel host threads) and, with load, load the code on the current
// device's context (without load nothing touches a device). On failure
// returns false with the compiler's log or the loader's error in err.
bool jit_compile(const Program &prog, JitProgram &out, std::string &err, bool load, bool df = false);

// Launch part i of a compiled program on the stream (grid: resident CTAs per
// SM times the SMs, at most one CTA per tile).
cudaError_t jit_launch(JitProgram &jp, size_t i, void *sv, uint64_t n_tiles, cudaStream_t st);

void jit_release(JitProgram &jp);

// Whether the run-time compiler could be loaded (and why not).
bool jit_available(std::string *why);

}  // namespace hisv
