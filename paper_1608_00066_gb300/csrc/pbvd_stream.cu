// Continuous streams decoded with carried path metrics (serving).
//
// A stream is decoded by Eq. (1) run once over all its stages, the metrics
// carried in device memory from one push to the next; segment m = [mD,
// (m+1)D) is released, once stage (m+1)D + L - 1 exists, by traceback from
// S_0 at that stage over its L + D records (the carried-metric window form of
// the oracle, for streams that never restart).  When the stream closes (its
// last v stages are the zero tail) the remaining stages are released by
// traceback from S_0 at the last stage.
//
// One launch serves many streams, one group of T threads per stream (lane A
// of the packed metrics; lane B is unused).  Every push processes whole
// periods of P stages (the host keeps the remainder for the next push), so
// the metrics are stored between pushes in the natural layout psi = u, and
// stage s always has phase s mod P.  Survivor records go to a per-stream
// ring of H records; the releases of one push are spread over the group's
// lanes.  Soft values are read straight from the caller's buffer; the stages
// of a partial period left at the end of a push are copied to the stream's
// carry buffer and decoded first by the next push.
#include "pbvd_device.cuh"

namespace pbvd {

template <class C, int T>
__device__ __forceinline__ void stream_push(const StreamDev& sd, uint32_t one, uint32_t* scratch) {
  using S = Shape<C, T>;
  constexpr int R = C::R, M = S::M, P = S::P, W = S::W, RW = S::RW;
  const int lane = threadIdx.x & 31;
  const int tau = lane & (T - 1);
  const unsigned gmask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
  const int nst = sd.ncarry + sd.nnew;
  const int nproc = sd.final_ ? nst : (nst / P) * P;
  const int64_t t0 = sd.t0;

  uint32_t pm[M];
#pragma unroll
  for (int k = 0; k < M; ++k) pm[k] = sd.pm[(tau << S::r) + k];
  uint32_t sel[P][3];
#pragma unroll
  for (int ph = 0; ph < P; ++ph) {
    const uint32_t m = thread_swap<C, T>(tau, ph);
#pragma unroll
    for (int q = 0; q < 3; ++q) sel[ph][q] = 0u - ((m >> (R - 1 - q)) & 1u);
  }
  PipeConsts pc;
  pc.one = one;
  pc.minus_one = 0u - one;

  int since_renorm = 0;
  for (int i0 = 0; i0 < nproc; i0 += P) {
#pragma unroll
    for (int ph = 0; ph < P; ++ph) {
      const int i = i0 + ph;
      if (i >= nproc) break;
      const int8_t* src = i < sd.ncarry ? sd.carry + i * R : sd.llr + (int64_t)(i - sd.ncarry) * R;
      uint32_t Pk[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) Pk[q] = q < R ? pack_soft((uint32_t)(uint8_t)src[q], 0u) : 0u;
      uint32_t bm[C::NC], kt[C::NC], wd[W];
      branch_metrics<C, (T > 1)>(Pk, sel[ph], bm, kt);
      if (ph == 0) acs_stage<C, T, 0>(pm, wd, bm, kt, pc);
      if constexpr (P > 1) if (ph == 1) acs_stage<C, T, (P > 1 ? 1 : 0)>(pm, wd, bm, kt, pc);
      if constexpr (P > 2) if (ph == 2) acs_stage<C, T, (P > 2 ? 2 : 0)>(pm, wd, bm, kt, pc);
      if constexpr (P > 3) if (ph == 3) acs_stage<C, T, (P > 3 ? 3 : 0)>(pm, wd, bm, kt, pc);
      if constexpr (P > 4) if (ph == 4) acs_stage<C, T, (P > 4 ? 4 : 0)>(pm, wd, bm, kt, pc);
      if constexpr (P > 5) if (ph == 5) acs_stage<C, T, (P > 5 ? 5 : 0)>(pm, wd, bm, kt, pc);
      if constexpr (P > 6) if (ph == 6) acs_stage<C, T, (P > 6 ? 6 : 0)>(pm, wd, bm, kt, pc);
      if constexpr (P > 7) if (ph == 7) acs_stage<C, T, (P > 7 ? 7 : 0)>(pm, wd, bm, kt, pc);
      uint32_t* rec = sd.ring + ((t0 + i) % sd.H) * RW + tau * W;
#pragma unroll
      for (int w = 0; w < W; ++w) rec[w] = wd[w];
    }
    if (i0 + P <= nproc) {
      if constexpr (T > 1) {
        __syncwarp(gmask);
#pragma unroll
        for (int k = 0; k < M; ++k) scratch[(k << S::t) | tau] = pm[k];
        __syncwarp(gmask);
#pragma unroll
        for (int k = 0; k < M; ++k) pm[k] = scratch[(tau << S::r) + k];
        __syncwarp(gmask);
      }
      if (++since_renorm == S::RENORM_PERIODS || i0 + P == nproc) {
        since_renorm = 0;
        uint32_t ref = pm[0];
        if constexpr (T > 1) ref = __shfl_sync(gmask, ref, 0, T);
#pragma unroll
        for (int k = 0; k < M; ++k) pm[k] = pm[k] + S::RENORM_BASE - ref;
      }
    }
  }
  if (!sd.final_) {
#pragma unroll
    for (int k = 0; k < M; ++k) sd.pm[(tau << S::r) + k] = pm[k];
  }
  __threadfence_block();
  __syncwarp(gmask);
  // the partial period left over becomes the next push's carry (when nothing
  // was decoded the carried stages stay where they are)
  for (int i = nproc + tau; i < nst; i += T)
    if (i >= sd.ncarry)
#pragma unroll
      for (int q = 0; q < R; ++q) sd.carry[(i - nproc) * R + q] = sd.llr[(int64_t)(i - sd.ncarry) * R + q];

  // releases: segments whose trigger stage exists, or everything at close
  const int64_t tend = t0 + nproc;
  const int64_t D = sd.D, L = sd.L;
  int64_t first = sd.released;
  int64_t nseg = 0;
  if (tend >= first + D + L) nseg = (tend - L - first) / D;  // (m+1)D + L - 1 <= tend - 1
  const bool last = sd.final_ != 0;
  const int64_t nwalk = nseg + ((last && first + nseg * D < tend) ? 1 : 0);
  for (int64_t w = tau; w < nwalk; w += T) {
    const int64_t lo = first + w * D;
    const bool is_tail = (w == nseg);
    const int64_t hi_out = is_tail ? tend : lo + D;  // exclusive
    const int64_t start = is_tail ? tend - 1 : lo + D + L - 1;
    int psi = 0;
    int lm = (1 << (int)(start % P)) - 1;
    uint32_t acc = 0u;
    for (int64_t s = start; s >= lo; --s) {
      const int bit = tb_step<C, T>(psi, lm, 0, sd.ring + (s % sd.H) * RW);
      acc = (acc << 1) | (uint32_t)bit;
      if ((s & 7) == 0 && s < hi_out) {
        const int64_t rem = hi_out - s;
        const uint32_t keep = rem >= 8 ? 0xffu : ((1u << rem) - 1u);
        sd.out[s >> 3] = (uint8_t)(acc & keep);
      }
    }
  }
}

template <class C, int T>
__global__ void __launch_bounds__(256, 1) pbvd_stream_kernel(const __grid_constant__ StreamLaunch p) {
  __shared__ __align__(16) uint32_t scratch[(256 / T) * (C::N + 4)];
  const int g = threadIdx.x / T;
  const int idx = blockIdx.x * (blockDim.x / T) + g;
  if (idx >= p.count) return;
  stream_push<C, T>(p.d[idx], p.one, scratch + g * (C::N + 4));
}

using K7 = Code<7, 0171u, 0133u, 0u>;
using K9 = Code<9, 0557u, 0663u, 0711u>;

template <class C, int T>
cudaError_t launch_stream(const StreamLaunch& p, int cta, cudaStream_t s) {
  if (cta < T || cta > 256 || cta % 32 != 0 || p.count <= 0 || p.count > kStreamsPerLaunch) return cudaErrorInvalidValue;
  const int groups = cta / T;
  const int grid = (p.count + groups - 1) / groups;
  pbvd_stream_kernel<C, T><<<grid, cta, 0, s>>>(p);
  return cudaGetLastError();
}

template <class C, int T>
StreamKernelEntry make_stream_entry() {
  StreamKernelEntry e;
  e.K = C::K;
  e.R = C::R;
  for (int r = 0; r < 3; ++r) e.gens[r] = C::gen(r);
  e.T = T;
  e.P = Shape<C, T>::P;
  e.words_per_stage = Shape<C, T>::RW;
  e.launch = &launch_stream<C, T>;
  return e;
}

int register_stream(StreamKernelEntry* out, int cap) {
  const StreamKernelEntry all[] = {make_stream_entry<K7, 8>(), make_stream_entry<K9, 8>()};
  int n = 0;
  for (const StreamKernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}

}  // namespace pbvd
