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
#include "pbvd_warp.cuh"

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


// ------------------------------------------------ one warp per K=7 stream --
//
// The 64-state streams run on the latency core of pbvd_warp.cuh: one warp
// per stream (lane A of the packed metrics; lane B unused), lane j owning
// butterfly j in natural state order, so every push decodes all its stages
// (a period of one stage: no carry).  Records go to the stream's ring in
// blocks of eight stages: stage t's decisions are in block (t >> 3) mod
// (H / 8), word u & 31 for state u, bit 16 (u >> 5) + (t & 7); lane j keeps
// the block's word in a register and stores it when the block is complete or
// the push ends (the next push reloads a partly filled word).  Each release
// walk prefetches whole blocks of 128 bytes into its lane's part of shared
// memory with cp.async.

constexpr int kStreamWarpSC = 64;      // stages per staged chunk
constexpr int kStreamWarpNB = 4;       // ring blocks in flight per walking lane

template <class C>
struct StreamWarpSmem {
  static constexpr int CB = ((kStreamWarpSC * C::R + 15) / 16 + 1) * 16;
  static constexpr int RAW_WORDS = 2 * CB / 4;
  static constexpr int TAB_WORDS = kStreamWarpSC * C::NC;
  static constexpr int WALK_WORDS = 32 * kStreamWarpNB * 32;
  static constexpr int WORDS = RAW_WORDS + TAB_WORDS + WALK_WORDS;
};

template <class C>
__device__ __forceinline__ void stream_warp_walk(const StreamDev& sd, int64_t start, int64_t lo, int64_t hi_out,
                                                 uint32_t* wring) {
  const int HB = sd.H >> 3;
  const int64_t b_top = start >> 3, b_lo = lo >> 3;
  const int nblk = (int)(b_top - b_lo + 1);
  int issued = 0;
  auto issue = [&]() {
    if (issued < nblk) {
      const int64_t b = b_top - issued;
      const uint32_t* src = sd.ring + (int64_t)(b % HB) * 32;
      const unsigned d = (unsigned)__cvta_generic_to_shared(wring + (issued % kStreamWarpNB) * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16 * q), "l"(src + 4 * q));
    }
    ++issued;
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int q = 0; q < kStreamWarpNB - 1; ++q) issue();
  uint32_t u = 0u, acc = 0u;
  int64_t t = start;
  for (int k = 0; k < nblk; ++k) {
    issue();
    asm volatile("cp.async.wait_group %0;" ::"n"(kStreamWarpNB - 1) : "memory");
    const uint32_t* blk = wring + (k % kStreamWarpNB) * 32;
    const int64_t tb = (b_top - k) << 3;   // first stage of the block
    for (; t >= tb && t >= lo; --t) {
      const uint32_t word = blk[u & 31u];
      const uint32_t upper = (word >> (16u * (u >> 5) + (uint32_t)(t & 7))) & 1u;
      acc = (acc << 1) | (u >> 5);
      u = ((u << 1) & 62u) | (upper ^ 1u);
      if ((t & 7) == 0 && t < hi_out) {
        const int64_t rem = hi_out - t;
        const uint32_t keep = rem >= 8 ? 0xffu : ((1u << rem) - 1u);
        sd.out[t >> 3] = (uint8_t)(acc & keep);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <class C>
__global__ void __launch_bounds__(32) pbvd_stream_warp_kernel(const __grid_constant__ StreamLaunch p) {
  static_assert(C::v == 6, "one butterfly per lane: 64 states");
  using SW = StreamWarpSmem<C>;
  constexpr int R = C::R, SC = kStreamWarpSC, CB = SW::CB;
  __shared__ __align__(16) uint32_t smem[SW::WORDS];
  const int idx = blockIdx.x;
  if (idx >= p.count) return;
  const StreamDev& sd = p.d[idx];
  const int lane = threadIdx.x & 31;
  int8_t* raw = reinterpret_cast<int8_t*>(smem);
  uint32_t* tab = smem + SW::RAW_WORDS;
  uint32_t* wring = smem + SW::RAW_WORDS + SW::TAB_WORDS + lane * (kStreamWarpNB * 32);

  const int nproc = sd.nnew;   // one-stage periods: every stage is decoded now
  const int64_t t0 = sd.t0;
  const int HB = sd.H >> 3;
  const uint32_t al = C::alpha((uint32_t)(2 * lane));
  uint32_t X = sd.pm[2 * lane], Y = sd.pm[2 * lane + 1];
  // the word of the block holding stage t0, partly filled by the last push
  uint32_t dacc = (t0 & 7) ? sd.ring[(int64_t)((t0 >> 3) % HB) * 32 + lane] : 0u;

  const int nchunk = (nproc + SC - 1) / SC;
  int64_t cb0 = stage_stream_chunk<R>(sd.llr, sd.nnew, 0, SC, raw, lane, 32);
  int64_t cb1 = 0;
  asm volatile("cp.async.commit_group;" ::: "memory");
  constexpr int RENORM = Shape<C, 1>::RENORM_STAGES;
  constexpr uint32_t RENORM_BASE = Shape<C, 1>::RENORM_BASE;
  int since_renorm = 0;
  for (int c = 0; c < nchunk; ++c) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    {
      const int8_t* buf = raw + (c & 1) * CB;
      const int64_t cbase = (c & 1) ? cb1 : cb0;
#pragma unroll
      for (int h = 0; h < SC / 32; ++h) {
        const int sl = lane + 32 * h;
        const int i = c * SC + sl;
        uint32_t pk[3] = {0u, 0u, 0u};
        if (i < nproc) {
          const uint8_t* src = reinterpret_cast<const uint8_t*>(buf) + ((int64_t)i * R - cbase);
#pragma unroll
          for (int q = 0; q < R; ++q) pk[q] = pack_soft(src[q], 0u);
        }
#pragma unroll
        for (int cw = 0; cw < C::NC; ++cw) {
          uint32_t m = 0u;
#pragma unroll
          for (int q = 0; q < R; ++q) m += ((cw >> (R - 1 - q)) & 1) ? pk[q] : kLamMax2 - pk[q];
          tab[sl * C::NC + cw] = m;
        }
      }
    }
    __syncwarp();
    if (c + 1 < nchunk) {
      const int64_t k0 = (int64_t)(c + 1) * SC;
      const int64_t cb = stage_stream_chunk<R>(sd.llr, sd.nnew, k0, k0 + SC, raw + ((c + 1) & 1) * CB, lane, 32);
      if ((c + 1) & 1) cb1 = cb; else cb0 = cb;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int iend = min(nproc, (c + 1) * SC);
    const int ic = c * SC;                               // first stage of the chunk
    const uint32_t* trow = tab + al;                     // trow[(i - ic) * NC]: stage i's metric
    auto renorm = [&]() {
      since_renorm = 0;
      const uint32_t ref = __shfl_sync(0xffffffffu, X, 0);  // state 0
      X = X + RENORM_BASE - ref;
      Y = Y + RENORM_BASE - ref;
    };
    auto step = [&](int i) {
      const uint32_t d = warp_acs<C>(X, Y, trow[(i - ic) * C::NC], lane);
      const int64_t t = t0 + i;
      const uint32_t col = 0x01010101u << (uint32_t)(t & 7);
      dacc = (dacc & ~col) | (d & col);
      if ((t & 7) == 7 || i == nproc - 1) sd.ring[(int64_t)((t >> 3) % HB) * 32 + lane] = dacc;
      if (++since_renorm == RENORM) renorm();
    };
    int i = c * SC;
    for (; i < iend && ((t0 + i) & 7) != 0; ++i) step(i);
    // whole blocks of eight stages (t = 8m .. 8m + 7) before the push's last
    // stage: no per-stage checks, the word stored once per block
    for (; i + 8 <= iend && i + 8 < nproc; i += 8) {
      if (since_renorm + 8 > RENORM) renorm();
      uint32_t bmv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) bmv[u] = trow[(i - ic + u) * C::NC];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t d = warp_acs<C>(X, Y, bmv[u], lane);
        const uint32_t col = 0x01010101u << u;
        dacc = (dacc & ~col) | (d & col);
      }
      sd.ring[(int64_t)(((t0 + i) >> 3) % HB) * 32 + lane] = dacc;
      since_renorm += 8;
    }
    for (; i < iend; ++i) step(i);
  }
  if (nproc > 0) {
    const uint32_t ref = __shfl_sync(0xffffffffu, X, 0);
    X = X + RENORM_BASE - ref;
    Y = Y + RENORM_BASE - ref;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!sd.final_) {
    sd.pm[2 * lane] = X;
    sd.pm[2 * lane + 1] = Y;
  }
  __threadfence_block();
  __syncwarp();

  // releases: segments whose trigger stage exists, or everything at close;
  // one walk per lane at a time
  const int64_t tend = t0 + nproc;
  const int64_t D = sd.D, L = sd.L;
  const int64_t first = sd.released;
  int64_t nseg = 0;
  if (tend >= first + D + L) nseg = (tend - L - first) / D;
  const bool last = sd.final_ != 0;
  const int64_t nwalk = nseg + ((last && first + nseg * D < tend) ? 1 : 0);
  for (int64_t w = lane; w < nwalk; w += 32) {
    const int64_t lo = first + w * D;
    const bool is_tail = (w == nseg);
    const int64_t hi_out = is_tail ? tend : lo + D;
    const int64_t start = is_tail ? tend - 1 : lo + D + L - 1;
    stream_warp_walk<C>(sd, start, lo, hi_out, wring);
  }
}

template <class C>
cudaError_t launch_stream_warp(const StreamLaunch& p, cudaStream_t s) {
  if (p.count <= 0 || p.count > kStreamsPerLaunch) return cudaErrorInvalidValue;
  pbvd_stream_warp_kernel<C><<<p.count, 32, 0, s>>>(p);
  return cudaGetLastError();
}

template <class C>
StreamKernelEntry make_stream_warp_entry() {
  StreamKernelEntry e;
  e.K = C::K;
  e.R = C::R;
  for (int r = 0; r < 3; ++r) e.gens[r] = C::gen(r);
  e.T = 32;
  e.P = 1;
  e.words_per_stage = 4;
  e.launch = &launch_stream_warp<C>;
  return e;
}

int register_stream(StreamKernelEntry* out, int cap) {
  const StreamKernelEntry all[] = {make_stream_warp_entry<K7>(), make_stream_entry<K9, 8>()};
  int n = 0;
  for (const StreamKernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}

}  // namespace pbvd
