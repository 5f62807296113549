// Decoding with 8-bit path metrics, four blocks per register (pbvd_pm8.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pbvd {

// The kernel instance and renormalisation interval for code (K, R, gens) on
// q-bit values with `lanes` threads per four blocks (0: the most built):
// pm8_plan returns -1 when no such instance is built or when K * 2QR >= 127
// (the metrics would not fit in bytes).
struct Pm8Plan {
  int inst;   // index of the kernel instance
  int q, Q;
  int bmmax;  // 2QR
  int rks;    // stages between renormalisations (K - 1: every rp periods)
  int rp;
  int lanes;  // threads per four blocks
};
int pm8_plan(int K, int R, const uint32_t* gens, int q, int lanes, Pm8Plan* p);

// Lock-step stages I, quads of blocks, and the words of the gathered values
// and of the survivor records of a stream of n stages.
void pm8_sizes(int K, int R, int64_t n, int D, int L, int64_t* I, int64_t* nquads, size_t* in_words,
               size_t* surv_words);

// Regroups the packed words into in (four blocks per word) and decodes into
// out; in and surv hold pm8_sizes' words.
cudaError_t pm8_launch(const Pm8Plan& p, int K, int R, const uint32_t* words, int64_t n, int D, int L,
                       uint32_t* in, uint32_t* surv, uint8_t* out, cudaStream_t s);

}  // namespace pbvd
