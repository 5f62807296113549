// Internal declarations shared by the host API and the kernel instances.
#pragma once

#ifdef __CUDACC_RTC__
#include "pbvd_rtc_types.h"
#else
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace pbvd {

// Argument block of every decode launch (passed by value).
struct KArgs {
  const int8_t* llr;      // soft values as sent
  uint8_t* out;           // packed decoded bits
  uint32_t* surv;         // global survivor records, [J][surv_pairs][surv_rs] words
  int64_t n;              // stages of the stream
  int64_t b_first;        // first block of this launch
  int64_t n_blocks;       // end (exclusive) of this launch's blocks; ceil(n / D) for a whole stream
  int64_t n_pairs;        // ceil((n_blocks - b_first) / 2)
  int64_t surv_pairs;     // pair slots per record row of surv
  int32_t surv_rs;        // words per record slot (>= the code's T*W record)
  int32_t pad_rs;
  int32_t D, L;
  int32_t smem_surv;      // 1: survivor records in shared memory
  int32_t smem_rec_words; // shared-memory record words per group (smem mode)
  int32_t punct_P;        // 0: not punctured, else pattern period
  int32_t punct_C;        // values sent per period
  int64_t llr_count;      // soft values readable at llr
  int32_t tb_argmin;      // 1: each block's traceback starts from its cheapest state (not S_0)
  int32_t circular;       // 1: tail-biting frame; llr holds stages [-L, n + L) wrapped around
  int16_t punct_off[32 * 4];  // [col][r]: offset in the period, -1 = punctured
  int16_t punct_pre[33];      // values sent in the columns before col
};

// Batched work: one entry per pair of PBs (each PB from its own frame).
struct BatchPair {
  const int8_t* llr[2];
  const int8_t* llr_end[2];
  uint8_t* out[2];
  int64_t n[2];       // stages of the frame
  int64_t b[2];       // block index within the frame
  int32_t hasB;
  int32_t pad;
};

// A tile: consecutive pairs of one code slot, one pair per group of a CTA.
struct BatchTile {
  int32_t slot;       // code slot of the combined kernel
  int32_t count;      // pairs in the tile
  int64_t first;      // index of the first pair
};

constexpr int kBatchSlots = 3;

struct BatchArgs {
  KArgs code[kBatchSlots];  // per code slot: D, L, puncture tables, survivors
  const BatchPair* pairs;
  const BatchTile* tiles;
  int32_t ntiles;
  int32_t gmax;             // survivor slots per CTA
  int32_t* counter;         // next tile to take (zeroed before the launch)
};

#ifndef __CUDACC_RTC__
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
  LaunchFn launch[2];      // [0]: records in the global workspace, [1]: in shared memory
  AttrFn set_max_smem[2];
  int jit;                 // -1: compiled into the library; else a kernel compiled at run time
  bool variants;           // the instance honouring KArgs::tb_argmin and KArgs::circular
};

#endif  // __CUDACC_RTC__

// One stream's push, as the stream kernel sees it.  The stages of the push
// are the ncarry stages held back from the previous push (carry buffer)
// followed by the nnew stages of the caller's buffer.
struct StreamDev {
  uint32_t* pm;          // N metric words (natural layout, lane A)
  uint32_t* ring;        // H survivor records of RW words
  int8_t* carry;         // up to P - 1 stages not yet decoded, R bytes each
  const int8_t* llr;     // the caller's new stages, R bytes each
  uint8_t* out;          // decoded bits of the whole stream
  int64_t t0;            // first stage of this push (multiple of P)
  int64_t released;      // first stage whose bits are not yet released
  int32_t ncarry, nnew;
  int32_t final_;        // 1: the stream ends here; decode and release all
  int32_t H;             // ring records
  int32_t D, L;
};

// Descriptors of up to kStreamsPerLaunch streams, passed by value as the
// kernel parameter (so a launch owns its descriptors and can be captured).
constexpr int kStreamsPerLaunch = 128;
struct StreamLaunch {
  int32_t count;
  StreamDev d[kStreamsPerLaunch];
};

#ifndef __CUDACC_RTC__
using StreamLaunchFn = cudaError_t (*)(const StreamLaunch& p, cudaStream_t s);

struct StreamKernelEntry {
  int K, R, T, P;
  uint32_t gens[3];
  int words_per_stage;
  StreamLaunchFn launch;
};

using BatchLaunchFn = cudaError_t (*)(const BatchArgs& a, int grid, int cta, size_t smem, cudaStream_t s);
using BatchOccFn = cudaError_t (*)(int* blocks_per_sm, int cta, size_t smem);
using BatchSlotLaunchFn = cudaError_t (*)(const BatchArgs& a, int slot, int grid, int cta, size_t smem, cudaStream_t s);
using BatchSlotOccFn = cudaError_t (*)(int slot, int* blocks_per_sm, int cta, size_t smem);
using BatchSlotAttrFn = cudaError_t (*)(int slot, int smem_bytes);

// The combined persistent kernel for mixed-code batches.
struct BatchKernelEntry {
  int K[kBatchSlots], R[kBatchSlots], T[kBatchSlots];
  uint32_t gens[kBatchSlots][3];
  bool punct[kBatchSlots];
  int words_per_stage[kBatchSlots];
  int scratch_words[kBatchSlots];
  BatchLaunchFn launch;
  AttrFn set_max_smem;
  BatchOccFn occupancy;
  // batches whose frames are all of one code slot: that slot's own kernel
  int single_T[kBatchSlots];
  int single_words_per_stage[kBatchSlots];
  int single_scratch_words[kBatchSlots];
  BatchSlotLaunchFn single_launch;
  BatchSlotAttrFn single_set_max_smem;
  BatchSlotOccFn single_occupancy;
};

// Unpacks q-bit soft values [v0, v1) of words into out[v0 .. v1) as int8,
// scaled to the decoder's range (pbvd_packed.cu).
cudaError_t launch_unpack(int q, const uint32_t* words, int64_t v0, int64_t v1, int8_t* out, cudaStream_t s);

// The paper's two-kernel design (pbvd_twokernel.cu): groups N_c of the code
// (-1 when the ablation is not built for it) and the launch of K1 and K2.
int two_kernel_groups(int K, int R, const uint32_t* gens);
cudaError_t two_kernel_launch(int K, const KArgs& a, uint32_t* sp, int64_t sp_pbs, cudaStream_t s);

// Registries filled by the instance files.
int register_k7(KernelEntry* out, int cap);
int register_k7_punctured(KernelEntry* out, int cap);
int register_k9(KernelEntry* out, int cap);
int register_small(KernelEntry* out, int cap);
int register_k7_r3(KernelEntry* out, int cap);
int register_batch(BatchKernelEntry* out, int cap);
int register_stream(StreamKernelEntry* out, int cap);

#endif  // __CUDACC_RTC__

}  // namespace pbvd
