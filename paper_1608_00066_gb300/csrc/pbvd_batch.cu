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
  decode_pair<C, T, PUNCT, false, false, false>(a, wk, slot, smem + g * SW, nullptr);
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

// Two shapes of the mixed-code kernel.  Wide (the default): K=7 paths at
// four threads per pair of blocks, K=9 at sixteen; its pairs are few and long
// in a batch of short frames, and more threads per pair shorten the chains
// that end the launch (measured fastest for the 10,000-frame mixed batch).
// Dense: K=7 at two threads per pair, K=9 at eight, fewer instructions per
// butterfly; faster where batches of long frames run several at a time and
// fill the GPU between them (the serving loop).
#define PBVD_BATCH_WIDE K7, 4, false, K7, 4, true, K9, 16, false
#define PBVD_BATCH_DENSE K7, 2, false, K7, 2, true, K9, 8, false

template <class C0, int T0, bool P0, class C1, int T1, bool P1, class C2, int T2, bool P2>
cudaError_t launch_batch(const BatchArgs& a, int grid, int cta, size_t smem, cudaStream_t s) {
  pbvd_batch_kernel<C0, T0, P0, C1, T1, P1, C2, T2, P2><<<grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C0, int T0, bool P0, class C1, int T1, bool P1, class C2, int T2, bool P2>
cudaError_t batch_max_smem(int bytes) {
  return cudaFuncSetAttribute(pbvd_batch_kernel<C0, T0, P0, C1, T1, P1, C2, T2, P2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class C0, int T0, bool P0, class C1, int T1, bool P1, class C2, int T2, bool P2>
cudaError_t batch_occupancy(int* blocks, int cta, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pbvd_batch_kernel<C0, T0, P0, C1, T1, P1, C2, T2, P2>,
                                                       cta, smem);
}

// Batches of a single code: one persistent kernel with only that code's
// path, so that it gets that path's register budget (MINB 64-thread CTAs
// per SM) instead of the largest of three.  K=7 r1/2 runs at two threads
// per pair with six CTAs per SM (168 registers): a batch of 10,000 frames
// then fits in about one wave (66 against 62 Gb/s at four threads per pair
// and eight CTAs, measured).
template <class C, int T, bool PUNCT, int MINB>
__global__ void __launch_bounds__(64, MINB) pbvd_batch_single_kernel(const BatchArgs b, const int slot) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(b.counter, 1);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= b.ntiles) break;
    const BatchTile t = b.tiles[tile];
    run_tile<C, T, PUNCT>(b.code[slot], b, t, smem);
  }
}

#define PBVD_SINGLE0 K7, 2, false, 6
#define PBVD_SINGLE1 K7, 4, true, 8
#define PBVD_SINGLE2 K9, 8, false, 8

cudaError_t launch_single(const BatchArgs& a, int slot, int grid, int cta, size_t smem, cudaStream_t s) {
  if (slot == 0)
    pbvd_batch_single_kernel<PBVD_SINGLE0><<<grid, cta, smem, s>>>(a, 0);
  else if (slot == 1)
    pbvd_batch_single_kernel<PBVD_SINGLE1><<<grid, cta, smem, s>>>(a, 1);
  else
    pbvd_batch_single_kernel<PBVD_SINGLE2><<<grid, cta, smem, s>>>(a, 2);
  return cudaGetLastError();
}

cudaError_t single_max_smem(int slot, int bytes) {
  if (slot == 0)
    return cudaFuncSetAttribute(pbvd_batch_single_kernel<PBVD_SINGLE0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
  if (slot == 1)
    return cudaFuncSetAttribute(pbvd_batch_single_kernel<PBVD_SINGLE1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
  return cudaFuncSetAttribute(pbvd_batch_single_kernel<PBVD_SINGLE2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t single_occupancy(int slot, int* blocks, int cta, size_t smem) {
  if (slot == 0)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pbvd_batch_single_kernel<PBVD_SINGLE0>, cta, smem);
  if (slot == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pbvd_batch_single_kernel<PBVD_SINGLE1>, cta, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pbvd_batch_single_kernel<PBVD_SINGLE2>, cta, smem);
}

template <class C, int T, bool P, int MINB>
void fill_single(BatchKernelEntry& e, int s) {
  e.single_T[s] = T;
  e.single_words_per_stage[s] = record_words_per_stage<C, T>();
  e.single_scratch_words[s] = scratch_words_per_group<C, T>();
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

template <class C0, int T0, bool P0, class C1, int T1, bool P1, class C2, int T2, bool P2>
BatchKernelEntry make_batch_entry() {
  BatchKernelEntry e;
  fill_slot<C0, T0, P0>(e, 0);
  fill_slot<C1, T1, P1>(e, 1);
  fill_slot<C2, T2, P2>(e, 2);
  e.launch = &launch_batch<C0, T0, P0, C1, T1, P1, C2, T2, P2>;
  e.set_max_smem = &batch_max_smem<C0, T0, P0, C1, T1, P1, C2, T2, P2>;
  e.occupancy = &batch_occupancy<C0, T0, P0, C1, T1, P1, C2, T2, P2>;
  fill_single<PBVD_SINGLE0>(e, 0);
  fill_single<PBVD_SINGLE1>(e, 1);
  fill_single<PBVD_SINGLE2>(e, 2);
  e.single_launch = &launch_single;
  e.single_set_max_smem = &single_max_smem;
  e.single_occupancy = &single_occupancy;
  return e;
}

// Entry 0: the wide shape (default); entry 1: the dense shape.
int register_batch(BatchKernelEntry* out, int cap) {
  int n = 0;
  if (n < cap) out[n++] = make_batch_entry<PBVD_BATCH_WIDE>();
  if (n < cap) out[n++] = make_batch_entry<PBVD_BATCH_DENSE>();
  return n;
}

}  // namespace pbvd
