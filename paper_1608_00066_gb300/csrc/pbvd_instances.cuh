// Helpers that turn a (code, T) kernel template into a registry entry.
#pragma once

#include "pbvd_device.cuh"

namespace pbvd {

template <class C, int T, bool PUNCT>
cudaError_t launch_decode(const KArgs& a, int grid, int cta, size_t smem, cudaStream_t s) {
  pbvd_decode_kernel<C, T, PUNCT><<<grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C, int T, bool PUNCT>
cudaError_t set_max_smem(int bytes) {
  return cudaFuncSetAttribute(pbvd_decode_kernel<C, T, PUNCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
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
  e.launch = &launch_decode<C, T, PUNCT>;
  e.set_max_smem = &set_max_smem<C, T, PUNCT>;
  return e;
}

}  // namespace pbvd
