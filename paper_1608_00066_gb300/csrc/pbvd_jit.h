// Run-time compiled decode kernels for codes the library has no built-in
// kernel for (see pbvd_jit.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pbvd_internal.h"

namespace pbvd {

// True when libnvrtc could be loaded.
bool jit_available();

// Writes up to cap entries (one per usable threads-per-pair value) for the
// code into out and returns how many; 0 without libnvrtc.  var: the instances
// that honour the traceback / frame variants.  Their kernels are compiled on
// first launch.
int jit_register(int K, int R, const uint32_t* gens, bool punct, bool var, KernelEntry* out, int cap);

// Launches (compiling first if needed) placement smem (0: survivors in the
// workspace, 1: in shared memory) of entry jit.  Returns a PBVD_* code.
int jit_launch(int jit, int smem, const KArgs& a, int grid, int cta, size_t smem_bytes, cudaStream_t s);

// Whether placement smem of entry jit is compiled and loaded already.
bool jit_loaded(int jit, int smem);

// Raises the kernel's dynamic shared-memory limit (compiling first if needed).
int jit_set_max_smem(int jit, int smem, int bytes);

// Text of the last failure of the functions above.
const char* jit_last_error();

}  // namespace pbvd
