// Internal declarations shared by the host API and the kernel instances.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pbvd {

// Argument block of every decode launch (passed by value).
struct KArgs {
  const int8_t* llr;      // soft values as sent
  uint8_t* out;           // packed decoded bits
  uint32_t* surv;         // global survivor records, [J][surv_pairs][T*W] words
  int64_t n;              // stages of the stream
  int64_t n_blocks;       // ceil(n / D)
  int64_t n_pairs;        // ceil(n_blocks / 2)
  int64_t surv_pairs;     // pair slots per record row of surv
  int32_t D, L;
  int32_t smem_surv;      // 1: survivor records in shared memory
  int32_t smem_rec_words; // shared-memory record words per group (smem mode)
  int32_t punct_P;        // 0: not punctured, else pattern period
  int32_t punct_C;        // values sent per period
  int64_t llr_count;      // soft values readable at llr
  uint32_t one;           // the value 1, opaque to the compiler (pipe balancing)
  int16_t punct_off[32 * 4];  // [col][r]: offset in the period, -1 = punctured
  int16_t punct_pre[33];      // values sent in the columns before col
};

// Batched work: one entry per pair of PBs.
struct BatchPair {
  const int8_t* llr;
  uint8_t* out;
  int64_t n;        // stages of the frame
  int64_t bA;       // first PB of the pair
  int32_t hasB;
  int32_t code;     // index into the batch's code table
};

struct BatchCode {
  int32_t D, L;
  int32_t punct_P, punct_C;
  int16_t punct_off[32 * 4];
};

using LaunchFn = cudaError_t (*)(const KArgs& a, int grid, int cta, size_t smem, cudaStream_t s);
using SmemFn = int (*)(int cta_threads, int smem_rec_words);  // dynamic smem bytes of a launch
using AttrFn = cudaError_t (*)(int smem_bytes);

// One compiled (code, T) instance.
struct KernelEntry {
  int K, R;
  uint32_t gens[3];
  int T;
  bool punct;              // built for punctured input
  int words_per_stage;     // survivor record words per stage per pair (T * W)
  int scratch_words;       // shared-memory words per group besides records
  LaunchFn launch;
  AttrFn set_max_smem;
};

// Registries filled by the instance files.
int register_k7(KernelEntry* out, int cap);
int register_k9(KernelEntry* out, int cap);
int register_small(KernelEntry* out, int cap);

}  // namespace pbvd
