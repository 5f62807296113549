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
// lanes.  Soft values are staged from the caller's buffer into shared memory
// by cp.async one 64-stage chunk ahead, and each traceback walk prefetches
// its survivor records a few at a time, so neither pass waits on a global
// load per stage.  The stages of a partial period left at the end of a push
// are copied to the stream's carry buffer and decoded first by the next push.
#include "pbvd_device.cuh"

namespace pbvd {

// Per-group shared memory of the stream kernel.
template <class C, int T>
struct StreamSmem {
  static constexpr int P = Shape<C, T>::P;
  static constexpr int SC = P * ((64 + P - 1) / P);         // stages per staged chunk
  static constexpr int CB = ((SC * C::R + 15) / 16 + 1) * 16;  // bytes per chunk buffer
  static constexpr int RW = Shape<C, T>::RW;
  static constexpr int KR = 4;                              // records per traceback prefetch
  static constexpr int NBUF = 3;                            // prefetch chunks in flight per lane
  static constexpr int TRANS_WORDS = C::N + 4;
  static constexpr int RAW_WORDS = 2 * CB / 4;
  static constexpr int RING_WORDS = T * NBUF * KR * RW;     // all lanes of the group
  static constexpr int WORDS = TRANS_WORDS + RAW_WORDS + RING_WORDS;
  static_assert((RW * 4) % 16 == 0, "records copied in 16-byte pieces");
};

// Stages soft values of new-stage indices [k0, k1) of the caller's buffer
// (R bytes each) into buf: 16-byte pieces inside the buffer by cp.async, the
// ragged edges by plain loads.  Returns the byte offset in the caller's
// buffer that byte 0 of buf holds.
template <int R>
__device__ __forceinline__ int64_t stage_stream_chunk(const int8_t* llr, int64_t nnew, int64_t k0, int64_t k1,
                                                      int8_t* buf, int lane, int nlanes) {
  if (k0 < 0) k0 = 0;
  if (k1 > nnew) k1 = nnew;
  if (k0 >= k1) return 0;
  const uintptr_t lo = reinterpret_cast<uintptr_t>(llr), hi = lo + (uintptr_t)(nnew * R);
  const uintptr_t first = lo + (uintptr_t)(k0 * R);
  const uintptr_t A0 = first & ~(uintptr_t)15;
  const uintptr_t A1 = lo + (uintptr_t)(k1 * R);
  const int npieces = (int)((A1 - A0 + 15) >> 4);
  for (int p = lane; p < npieces; p += nlanes) {
    const uintptr_t src = A0 + ((uintptr_t)p << 4);
    int8_t* dst = buf + (p << 4);
    if (src >= lo && src + 16 <= hi) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src));
    } else {
      for (int q = 0; q < 16; ++q)
        if (src + q >= lo && src + q < hi) dst[q] = *reinterpret_cast<const int8_t*>(src + q);
    }
  }
  return (int64_t)(A0 - lo);
}

// One traceback walk: records s = start down to lo of the stream's ring,
// prefetched by cp.async KR at a time into this lane's ring in shared memory;
// emits the decoded bits of stages [lo, hi_out) as whole bytes.
template <class C, int T>
__device__ __forceinline__ void stream_walk(const StreamDev& sd, int64_t start, int64_t lo, int64_t hi_out,
                                            uint32_t* lring) {
  using SS = StreamSmem<C, T>;
  constexpr int P = Shape<C, T>::P, RW = SS::RW, KR = SS::KR, NBUF = SS::NBUF;
  const int nrec = (int)(start - lo + 1);
  const int nchunk = (nrec + KR - 1) / KR;
  const int H = sd.H;
  int ipos = (int)(start % H);   // ring position of the next record to request
  int issued = 0;
  auto issue = [&]() {
    if (issued < nchunk) {
      uint32_t* dst0 = lring + (issued % NBUF) * (KR * RW);
#pragma unroll
      for (int q = 0; q < KR; ++q) {
        if (issued * KR + q < nrec) {
          const uint32_t* src = sd.ring + (int64_t)ipos * RW;
          ipos = ipos == 0 ? H - 1 : ipos - 1;
          const unsigned d = (unsigned)__cvta_generic_to_shared(dst0 + q * RW);
#pragma unroll
          for (int w = 0; w < RW; w += 4)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 4 * w), "l"(src + w));
        }
      }
    }
    ++issued;
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int q = 0; q < NBUF - 1; ++q) issue();
  int psi = 0;
  int lm = (1 << (int)(start % P)) - 1;
  uint32_t acc = 0u;
  for (int ch = 0; ch < nchunk; ++ch) {
    issue();
    asm volatile("cp.async.wait_group %0;" ::"n"(NBUF - 1) : "memory");
    const uint32_t* buf = lring + (ch % NBUF) * (KR * RW);
    const int64_t top = start - ch * KR;
#pragma unroll
    for (int q = 0; q < KR; ++q) {
      const int64_t s = top - q;
      if (s >= lo) {
        const int bit = tb_step<C, T>(psi, lm, 0, buf + q * RW);
        acc = (acc << 1) | (uint32_t)bit;
        if ((s & 7) == 0 && s < hi_out) {
          const int64_t rem = hi_out - s;
          const uint32_t keep = rem >= 8 ? 0xffu : ((1u << rem) - 1u);
          sd.out[s >> 3] = (uint8_t)(acc & keep);
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <class C, int T>
__device__ __forceinline__ void stream_push(const StreamDev& sd, uint32_t* smem) {
  using S = Shape<C, T>;
  using SS = StreamSmem<C, T>;
  constexpr int R = C::R, M = S::M, P = S::P, W = S::W, RW = S::RW, SC = SS::SC, CB = SS::CB;
  const int lane = threadIdx.x & 31;
  const int tau = lane & (T - 1);
  const unsigned gmask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
  const int nst = sd.ncarry + sd.nnew;
  const int nproc = sd.final_ ? nst : (nst / P) * P;
  const int64_t t0 = sd.t0;
  uint32_t* scratch = smem;
  int8_t* raw = reinterpret_cast<int8_t*>(smem + SS::TRANS_WORDS);
  uint32_t* lring = smem + SS::TRANS_WORDS + SS::RAW_WORDS + tau * (SS::NBUF * SS::KR * RW);

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

  // chunk c holds stages [c SC, (c + 1) SC) of the push; stage i >= ncarry
  // is new stage i - ncarry of the caller's buffer
  const int nchunk = (nproc + SC - 1) / SC;
  int64_t cb0 = stage_stream_chunk<R>(sd.llr, sd.nnew, -(int64_t)sd.ncarry, SC - sd.ncarry, raw, tau, T);
  int64_t cb1 = 0;
  asm volatile("cp.async.commit_group;" ::: "memory");

  const int H = sd.H;
  int rpos = (int)(t0 % H);      // ring position of the next record
  int since_renorm = 0;
  for (int i0 = 0; i0 < nproc; i0 += P) {
    if (i0 % SC == 0) {
      const int c = i0 / SC;
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp(gmask);
      if (c + 1 < nchunk) {
        const int nb = (c + 1) & 1;
        const int64_t k0 = (int64_t)(c + 1) * SC - sd.ncarry;
        const int64_t cb = stage_stream_chunk<R>(sd.llr, sd.nnew, k0, k0 + SC, raw + nb * CB, tau, T);
        if (nb) cb1 = cb; else cb0 = cb;
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int cur = (i0 / SC) & 1;
    const int8_t* buf = raw + cur * CB;
    const int64_t cbase = cur ? cb1 : cb0;
#pragma unroll
    for (int ph = 0; ph < P; ++ph) {
      const int i = i0 + ph;
      if (i >= nproc) break;
      const int8_t* src = i < sd.ncarry ? sd.carry + i * R : buf + ((int64_t)(i - sd.ncarry) * R - cbase);
      uint32_t Pk[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) Pk[q] = q < R ? pack_soft((uint32_t)(uint8_t)src[q], 0u) : 0u;
      uint32_t bm[C::NC], kt[C::NC], wd[W];
      branch_metrics<C, (T > 1)>(Pk, sel[ph], bm, kt);
      if (ph == 0) acs_stage<C, T, 0>(pm, wd, bm, kt);
      if constexpr (P > 1) if (ph == 1) acs_stage<C, T, (P > 1 ? 1 : 0)>(pm, wd, bm, kt);
      if constexpr (P > 2) if (ph == 2) acs_stage<C, T, (P > 2 ? 2 : 0)>(pm, wd, bm, kt);
      if constexpr (P > 3) if (ph == 3) acs_stage<C, T, (P > 3 ? 3 : 0)>(pm, wd, bm, kt);
      if constexpr (P > 4) if (ph == 4) acs_stage<C, T, (P > 4 ? 4 : 0)>(pm, wd, bm, kt);
      if constexpr (P > 5) if (ph == 5) acs_stage<C, T, (P > 5 ? 5 : 0)>(pm, wd, bm, kt);
      if constexpr (P > 6) if (ph == 6) acs_stage<C, T, (P > 6 ? 6 : 0)>(pm, wd, bm, kt);
      if constexpr (P > 7) if (ph == 7) acs_stage<C, T, (P > 7 ? 7 : 0)>(pm, wd, bm, kt);
      uint32_t* rec = sd.ring + (int64_t)rpos * RW + tau * W;
      rpos = rpos + 1 == H ? 0 : rpos + 1;
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
  asm volatile("cp.async.wait_group 0;" ::: "memory");
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

  // releases: segments whose trigger stage exists, or everything at close;
  // one walk per lane at a time
  const int64_t tend = t0 + nproc;
  const int64_t D = sd.D, L = sd.L;
  const int64_t first = sd.released;
  int64_t nseg = 0;
  if (tend >= first + D + L) nseg = (tend - L - first) / D;  // (m+1)D + L - 1 <= tend - 1
  const bool last = sd.final_ != 0;
  const int64_t nwalk = nseg + ((last && first + nseg * D < tend) ? 1 : 0);
  for (int64_t w = tau; w < nwalk; w += T) {
    const int64_t lo = first + w * D;
    const bool is_tail = (w == nseg);
    const int64_t hi_out = is_tail ? tend : lo + D;  // exclusive
    const int64_t start = is_tail ? tend - 1 : lo + D + L - 1;
    stream_walk<C, T>(sd, start, lo, hi_out, lring);
  }
}

// The stream kernel runs one warp per CTA: kStreamCta / T streams.
constexpr int kStreamCta = 32;

template <class C, int T>
__global__ void __launch_bounds__(kStreamCta) pbvd_stream_kernel(const __grid_constant__ StreamLaunch p) {
  __shared__ __align__(16) uint32_t smem[(kStreamCta / T) * StreamSmem<C, T>::WORDS];
  const int g = threadIdx.x / T;
  const int idx = blockIdx.x * (kStreamCta / T) + g;
  if (idx >= p.count) return;
  stream_push<C, T>(p.d[idx], smem + g * StreamSmem<C, T>::WORDS);
}

using K7 = Code<7, 0171u, 0133u, 0u>;
using K9 = Code<9, 0557u, 0663u, 0711u>;

template <class C, int T>
cudaError_t launch_stream(const StreamLaunch& p, cudaStream_t s) {
  if (p.count <= 0 || p.count > kStreamsPerLaunch) return cudaErrorInvalidValue;
  const int groups = kStreamCta / T;
  const int grid = (p.count + groups - 1) / groups;
  pbvd_stream_kernel<C, T><<<grid, kStreamCta, 0, s>>>(p);
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
