// Persistent kernel for batches of frames of mixed codes: K=7 (171,133)
// rate 1/2, the same code punctured, and K=9 (557,663,711) rate 1/3, all in
// one launch.  CTAs take tiles of pairs from an atomic counter; a tile holds
// pairs of one code and the CTA's threads form groups of that code's T.
#include "pbvd_instances.cuh"

namespace pbvd {

using K7 = Code<7, 0171u, 0133u, 0u>;
using K9 = Code<9, 0557u, 0663u, 0711u>;

template <class C, int T, bool PUNCT>
__device__ __forceinline__ void run_tile(const KArgs& a, const BatchArgs& b, const BatchTile& t, uint32_t* smem) {
  const int g = threadIdx.x / T;
  if (g >= t.count) return;
  const BatchPair& p = b.pairs[t.first + g];
  PairWork wk;
  wk.A.llr = p.llr[0];
  wk.A.llr_end = p.llr_end[0];
  wk.A.out = p.out[0];
  wk.A.n = p.n[0];
  wk.A.b = p.b[0];
  wk.B.llr = p.llr[1];
  wk.B.llr_end = p.llr_end[1];
  wk.B.out = p.out[1];
  wk.B.n = p.n[1];
  wk.B.b = p.b[1];
  wk.hasB = p.hasB != 0;
  constexpr int SW = scratch_words_per_group<C, T>();
  const int64_t slot = (int64_t)blockIdx.x * b.gmax + g;
  decode_pair<C, T, PUNCT, false>(a, wk, slot, smem + g * SW, nullptr);
}

template <class C0, int T0, bool P0, class C1, int T1, bool P1, class C2, int T2, bool P2>
__global__ void __launch_bounds__(256, 1) pbvd_batch_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(b.counter, 1);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= b.ntiles) break;
    const BatchTile t = b.tiles[tile];
    if (t.slot == 0)
      run_tile<C0, T0, P0>(b.code[0], b, t, smem);
    else if (t.slot == 1)
      run_tile<C1, T1, P1>(b.code[1], b, t, smem);
    else
      run_tile<C2, T2, P2>(b.code[2], b, t, smem);
  }
}

#define PBVD_BATCH_ARGS K7, 2, false, K7, 2, true, K9, 8, false

cudaError_t launch_batch(const BatchArgs& a, int grid, int cta, size_t smem, cudaStream_t s) {
  pbvd_batch_kernel<PBVD_BATCH_ARGS><<<grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t batch_max_smem(int bytes) {
  return cudaFuncSetAttribute(pbvd_batch_kernel<PBVD_BATCH_ARGS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t batch_occupancy(int* blocks, int cta, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pbvd_batch_kernel<PBVD_BATCH_ARGS>, cta, smem);
}

template <class C, int T, bool P>
void fill_slot(BatchKernelEntry& e, int s) {
  e.K[s] = C::K;
  e.R[s] = C::R;
  e.T[s] = T;
  for (int r = 0; r < 3; ++r) e.gens[s][r] = C::gen(r);
  e.punct[s] = P;
  e.words_per_stage[s] = record_words_per_stage<C, T>();
  e.scratch_words[s] = scratch_words_per_group<C, T>();
}

int register_batch(BatchKernelEntry* out, int cap) {
  if (cap < 1) return 0;
  BatchKernelEntry e;
  fill_slot<K7, 2, false>(e, 0);
  fill_slot<K7, 2, true>(e, 1);
  fill_slot<K9, 8, false>(e, 2);
  e.launch = &launch_batch;
  e.set_max_smem = &batch_max_smem;
  e.occupancy = &batch_occupancy;
  out[0] = e;
  return 1;
}

}  // namespace pbvd
