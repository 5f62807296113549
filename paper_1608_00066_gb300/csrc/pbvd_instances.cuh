// Helpers that turn a (code, T) kernel template into a registry entry.
#pragma once

#include "pbvd_device.cuh"
#include "pbvd_warp.cuh"

namespace pbvd {

template <class C, int T, bool PUNCT, bool SMEM>
cudaError_t launch_decode(const KArgs& a, int grid, int cta, size_t smem, cudaStream_t s) {
  pbvd_decode_kernel<C, T, PUNCT, SMEM><<<grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C, int T, bool PUNCT, bool SMEM>
cudaError_t set_max_smem(int bytes) {
  return cudaFuncSetAttribute(pbvd_decode_kernel<C, T, PUNCT, SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

template <class C, int T, bool PUNCT = false>
KernelEntry make_entry() {
  KernelEntry e;
  e.K = C::K;
  e.R = C::R;
  e.gens[0] = C::gen(0);
  e.gens[1] = C::gen(1);
  e.gens[2] = C::gen(2);
  e.T = T;
  e.punct = PUNCT;
  e.words_per_stage = record_words_per_stage<C, T>();
  e.scratch_words = scratch_words_per_group<C, T>();
  e.launch[0] = &launch_decode<C, T, PUNCT, false>;
  e.launch[1] = &launch_decode<C, T, PUNCT, true>;
  e.set_max_smem[0] = &set_max_smem<C, T, PUNCT, false>;
  e.set_max_smem[1] = &set_max_smem<C, T, PUNCT, true>;
  e.jit = -1;
  e.variants = false;
  return e;
}

template <class C, bool PUNCT, bool SMEM>
cudaError_t launch_warp(const KArgs& a, int grid, int cta, size_t smem, cudaStream_t s) {
  pbvd_warp_kernel<C, PUNCT, SMEM><<<grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C, bool PUNCT, bool SMEM>
cudaError_t set_max_smem_warp(int bytes) {
  return cudaFuncSetAttribute(pbvd_warp_kernel<C, PUNCT, SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// The latency kernel (one warp per pair of PBs, pbvd_warp.cuh) as the
// 32-threads-per-pair entry of a 64-state code: four-word records in natural
// state order.
template <class C, bool PUNCT = false>
KernelEntry make_warp_entry() {
  KernelEntry e;
  e.K = C::K;
  e.R = C::R;
  e.gens[0] = C::gen(0);
  e.gens[1] = C::gen(1);
  e.gens[2] = C::gen(2);
  e.T = 32;
  e.punct = PUNCT;
  e.words_per_stage = 4;
  e.scratch_words = warp_scratch_words<C>();
  e.launch[0] = &launch_warp<C, PUNCT, false>;
  e.launch[1] = &launch_warp<C, PUNCT, true>;
  e.set_max_smem[0] = &set_max_smem_warp<C, PUNCT, false>;
  e.set_max_smem[1] = &set_max_smem_warp<C, PUNCT, true>;
  e.jit = -1;
  e.variants = false;
  return e;
}

}  // namespace pbvd
