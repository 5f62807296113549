// 8-bit path metrics: four parallel blocks per 32-bit register (Sec. IV-C's
// q-bit soft values with small q).
//
// Branch metrics.  On q-bit values the metric of Sec. II is
// BM(c) = sum_r |lambda_r - mu(c_r)| with mu = +-Q, Q = 2^{q-1} - 1 (Q = 1 for
// hard decisions), values below -Q read as -Q; with a_r = lambda_r + Q in
// [0, 2Q] it is sum_r (c_r ? a_r : 2Q - a_r), at most BMmax = 2QR.
//
// Why 8 bits suffice.  Every state is reached from every state of v = K - 1
// stages earlier along some path of v branches, so after the first v stages
// (or from all-zero start metrics at once) every metric of a block lies within
// v BMmax of the block's smallest one, and the smallest one grows by at most
// BMmax per stage.  If the smallest metric is subtracted from all of them
// (renormalisation) at least every k stages, a candidate PM + BM never exceeds
// (k - 1 + K) BMmax; with that at most 127 every candidate is a 7-bit value:
// - a plain 32-bit add of two registers adds the four byte lanes without a
//   carry between them;
// - y + 0x80 - x (per byte, again one 32-bit operation) lies in [1, 255], so
//   bit 7 of each byte is (y >= x), and the sign-replicating byte permute
//   turns it into a 0x00 / 0xFF mask that selects the smaller candidate and
//   is itself the decision bit.
// Subtracting the same value from every metric of a block changes no
// decision, so the decoded bits are those of the exact integer metric
// (ties included: the upper branch is kept when c1 >= c0, as Eq. (1) with
// the lower-index tie rule does).
//
// Known start (a block whose range begins at stage 0): states other than S_0
// start at BIG = 127 - BMmax, and during the first v stages every state that
// S_0 cannot have reached yet is set to BIG again after its stage.  A
// reachable candidate is at most v BMmax < BIG, so no reachable state ever
// takes an unreachable predecessor, and the traceback (from S_0, along
// reachable states only) reads none of the decisions of unreachable states.
//
// Layout: a quad of four consecutive blocks 4q .. 4q+3, block l in byte l of
// every register, is decoded by one thread (pm8_decode_kernel) or by two
// that split its states (pm8_decode2_kernel, 64-state codes); the quad runs
// in lock step over I = min(D + 2L, n)
// stages, each block over its own [f0, f1] from stage index 0, padded with
// neutral values (a = Q: every codeword the same metric) after its end.  A
// gather kernel first writes the biased values of the four blocks of every
// quad and stage as one 32-bit word per code bit, so that the decoder's loads
// are coalesced.  The add-compare-select runs on the logical state array in
// a loop unrolled over one period of v stages (the successor of the register
// pair (2j, 2j+1) is (j, j + N/2): a rotation of the state index, which
// returns to the start after v stages, so the compiler keeps every metric in
// place).  Survivor records: per stage and quad N/8 words, word w bit 8l + k =
// 1 iff state 8w + k of block l kept its upper predecessor S_{2j}.  The
// traceback walks the chains (four per thread, or two per lane of a pair)
// over records staged in a per-thread shared-memory ring (cp.async).
#include <cstdint>
#include <cuda_runtime.h>

#include "pbvd_pm8.h"

namespace pbvd {
namespace {

constexpr uint32_t kByteSign = 0x80808080u;

// Codeword c(S_d, x) of Eq. (2), c^(1) most significant: bit r of the
// transition's register (x << (K-1)) | d filtered by generator r.
__host__ __device__ constexpr uint32_t cw_of(int K, int R, uint32_t g0, uint32_t g1, uint32_t g2, uint32_t d,
                                             uint32_t x) {
  const uint32_t reg = (x << (K - 1)) | d;
  uint32_t c = 0;
  for (int r = 0; r < R; ++r) {
    const uint32_t g = r == 0 ? g0 : (r == 1 ? g1 : g2);
    uint32_t p = g & reg, par = 0;
    while (p) {
      par ^= p & 1u;
      p >>= 1;
    }
    c = (c << 1) | par;
  }
  return c;
}

template <int K_, uint32_t G0, uint32_t G1, uint32_t G2>
struct Pm8Code {
  static constexpr int v = K_ - 1;
  static constexpr int N = 1 << v;
  static constexpr int H = N / 2;
  static constexpr int R = G2 ? 3 : 2;
  static constexpr int W = N / 8;  // record words per stage of a quad
  __host__ __device__ static constexpr uint32_t cw(uint32_t d, uint32_t x) { return cw_of(K_, R, G0, G1, G2, d, x); }
};

__device__ __forceinline__ uint32_t sign_mask(uint32_t d) {
  uint32_t m;
  asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(m) : "r"(d));
  return m;
}

// Per byte: the smaller of x and y (both in [0, 127]).
__device__ __forceinline__ uint32_t byte_min(uint32_t x, uint32_t y) {
  const uint32_t m = sign_mask(y + kByteSign - x);  // 0xFF where y >= x
  return (x & m) | (y & ~m);
}


struct Pm8Args {
  const uint32_t* in;  // biased values: word (i * nquads + q) * R + r, byte l = block 4q + l
  uint32_t* surv;      // records: words (i * nquads + q) * W .. + W
  uint8_t* out;        // decoded bits, LSB first
  int64_t n;           // stages
  int64_t nb;          // blocks
  int64_t nquads;
  int D, L, I;         // I: lock-step stages of every quad
  int rp;              // periods between renormalisations (interval = v)
  uint32_t big4;       // 127 - BMmax in every byte
  uint32_t twoq4;      // 2Q in every byte
};

// Geometry of block b in the quad's lock-step index (index 0 = stage f0).
struct Pm8Pb {
  int64_t f0;
  int len;  // f1 - f0 + 1 (0: no such block)
  int ob;   // first output stage bD - f0
  int oe;   // end of output min((b+1)D, n) - f0
};

__host__ __device__ __forceinline__ Pm8Pb pm8_pb(const Pm8Args& a, int64_t b) {
  Pm8Pb p{0, 0, 0, 0};
  if (b >= a.nb) return p;
  const int64_t s = b * a.D - a.L, e = (b + 1) * a.D + a.L;
  p.f0 = s < 0 ? 0 : s;
  const int64_t f1 = (e < a.n ? e : a.n) - 1;
  const int64_t o1 = (b + 1) * a.D < a.n ? (b + 1) * a.D : a.n;
  p.len = (int)(f1 - p.f0 + 1);
  p.ob = (int)(b * a.D - p.f0);
  p.oe = (int)(o1 - p.f0);
  return p;
}

// The biased values a = lambda + Q (lambda clamped at -Q) of the four blocks
// of a quad, one word per stage and code bit; a = Q (lambda = 0, the same
// metric for every codeword) past a block's end.  Thread: one quad, 32
// stages; each block's values are read in order, the word and the position
// in it advanced value by value.
template <int Q_BITS>
__global__ void __launch_bounds__(256) pm8_gather_kernel(const uint32_t* __restrict__ words, const Pm8Args a, int R,
                                                         uint32_t* __restrict__ in) {
  constexpr int M = 32 / Q_BITS;
  constexpr int QM = Q_BITS == 1 ? 1 : (1 << (Q_BITS - 1)) - 1;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nquads) return;
  const int i0 = blockIdx.y * 32;
  const int i1 = i0 + 32 < a.I ? i0 + 32 : a.I;
  int len[4];
  int64_t wi[4];   // word holding the block's next value
  int slot[4];     // position of that value in the word
  uint32_t cur[4]; // that word
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const Pm8Pb p = pm8_pb(a, 4 * q + l);
    len[l] = p.len;
    const int64_t idx = (p.f0 + i0) * R;
    wi[l] = idx / M;
    slot[l] = (int)(idx - wi[l] * M);
    cur[l] = i0 < p.len ? __ldg(words + wi[l]) : 0u;
  }
  for (int i = i0; i < i1; ++i) {
    for (int r = 0; r < R; ++r) {
      uint32_t acc = 0;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        int val = QM;
        if (i < len[l]) {
          const uint32_t u = (cur[l] >> (Q_BITS * slot[l])) & ((1u << Q_BITS) - 1u);
          int lam;
          if (Q_BITS == 1) {
            lam = u ? -1 : 1;
          } else {
            lam = (int)u - (int)((u >> (Q_BITS - 1)) << Q_BITS);  // sign-extend
            lam = lam < -QM ? -QM : lam;
          }
          val = lam + QM;
          if (++slot[l] == M) {
            slot[l] = 0;
            ++wi[l];
            // the next word, if the block has a value left in it
            const int64_t left = (int64_t)(len[l] - i) * R - r - 1;
            if (left > 0) cur[l] = __ldg(words + wi[l]);
          }
        }
        acc |= (uint32_t)val << (8 * l);
      }
      in[((int64_t)i * a.nquads + q) * R + r] = acc;
    }
  }
}

// Packs eight 0x00 / 0xFF byte masks into one word: bit k of byte l is byte l
// of mask LO + k (selects with constants, as the masks are all-zero or
// all-one bytes).
template <int LO, int NM>
__device__ __forceinline__ uint32_t merge_masks(const uint32_t* m) {
  if constexpr (NM == 1) {
    return m[LO];
  } else {
    const uint32_t lo = merge_masks<LO, NM / 2>(m);
    const uint32_t hi = merge_masks<LO + NM / 2, NM / 2>(m);
    constexpr uint32_t sel = ((((1u << (NM / 2)) - 1u) << (NM / 2)) << (LO & 7)) * 0x01010101u;
    return (lo & ~sel) | (hi & sel);
  }
}

// Subtracts the smallest metric of each byte lane from all metrics.
template <int N>
__device__ __forceinline__ void renormalise(uint32_t (&pm)[N]) {
  uint32_t t[N / 2];
#pragma unroll
  for (int j = 0; j < N / 2; ++j) t[j] = byte_min(pm[2 * j], pm[2 * j + 1]);
#pragma unroll
  for (int w = N / 4; w >= 1; w /= 2)
#pragma unroll
    for (int j = 0; j < w; ++j) t[j] = byte_min(t[2 * j], t[2 * j + 1]);
#pragma unroll
  for (int s = 0; s < N; ++s) pm[s] -= t[0];
}

// RKS: stages between renormalisations when it is below v; RKS = v means
// every a.rp periods.
template <class C, int RKS>
__global__ void __launch_bounds__(32) pm8_decode_kernel(const Pm8Args a) {
  constexpr int v = C::v, N = C::N, H = C::H, R = C::R, W = C::W;
  constexpr int NCW = 1 << R;
  constexpr int CS = 8, RB = 4;  // traceback ring: stages per chunk, chunks
  static_assert(v % RKS == 0, "renormalisation interval divides the period");
  static_assert(W >= 2 && W % 2 == 0, "at least 16 states");
  extern __shared__ __align__(16) uint32_t pm8_ring[];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nquads) return;
  Pm8Pb pb[4];
  uint32_t kmask = 0;  // 0xFF in the bytes of blocks with a known start
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    pb[l] = pm8_pb(a, 4 * q + l);
    if (pb[l].len > 0 && pb[l].f0 == 0) kmask |= 0xFFu << (8 * l);
  }
  uint32_t pm[N];
  pm[0] = 0;
#pragma unroll
  for (int s = 1; s < N; ++s) pm[s] = a.big4 & kmask;

  const int64_t in_stride = a.nquads * R, sv_stride = a.nquads * W;
  const uint32_t* inp = a.in + q * R;
  uint32_t* svp = a.surv + q * W;
  int per = 0;
  for (int i0 = 0; i0 < a.I; i0 += v) {
    uint32_t x[v][R];
#pragma unroll
    for (int p = 0; p < v; ++p)
#pragma unroll
      for (int r = 0; r < R; ++r) x[p][r] = (i0 + p < a.I) ? __ldg(inp + (int64_t)(i0 + p) * in_stride + r) : 0u;
#pragma unroll
    for (int p = 0; p < v; ++p) {
      if (i0 + p >= a.I) break;
      uint32_t cmp[R], bm[NCW];
#pragma unroll
      for (int r = 0; r < R; ++r) cmp[r] = a.twoq4 - x[p][r];
#pragma unroll
      for (int c = 0; c < NCW; ++c) {
        uint32_t t = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) t += ((c >> (R - 1 - r)) & 1) ? x[p][r] : cmp[r];
        bm[c] = t;
      }
      uint32_t nw[N], mk[N];
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const uint32_t u0 = pm[2 * j], u1 = pm[2 * j + 1];
#pragma unroll
        for (int xb = 0; xb < 2; ++xb) {
          const uint32_t c0 = u0 + bm[C::cw(2 * j, xb)];
          const uint32_t c1 = u1 + bm[C::cw(2 * j + 1, xb)];
          const uint32_t m = sign_mask(c1 + kByteSign - c0);  // 0xFF: c1 >= c0, upper kept
          nw[j + xb * H] = (c0 & m) | (c1 & ~m);
          mk[j + xb * H] = m;
        }
      }
      if (i0 == 0 && kmask) {
        // states S_0 has not reached after p + 1 stages: low v - p - 1 bits set
#pragma unroll
        for (int s = 1; s < N; ++s)
          if (s & ((1 << (v - p - 1)) - 1)) nw[s] = (nw[s] & ~kmask) | (a.big4 & kmask);
      }
      uint32_t rec[W];
#pragma unroll
      for (int w = 0; w < W; ++w) rec[w] = merge_masks<0, 8>(mk + 8 * w);
      uint32_t* dst = svp + (int64_t)(i0 + p) * sv_stride;
      if constexpr (W % 4 == 0) {
#pragma unroll
        for (int w = 0; w < W; w += 4)
          *reinterpret_cast<uint4*>(dst + w) = make_uint4(rec[w], rec[w + 1], rec[w + 2], rec[w + 3]);
      } else {
#pragma unroll
        for (int w = 0; w < W; w += 2) *reinterpret_cast<uint2*>(dst + w) = make_uint2(rec[w], rec[w + 1]);
      }
#pragma unroll
      for (int s = 0; s < N; ++s) pm[s] = nw[s];
      if constexpr (RKS < v) {
        if ((p + 1) % RKS == 0) renormalise<N>(pm);
      } else {
        if (p == v - 1 && ++per == a.rp) {
          per = 0;
          renormalise<N>(pm);
        }
      }
    }
  }

  // traceback of the four blocks from S_0 at their last stages
  int imin = a.I;
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (pb[l].len > 0 && pb[l].ob < imin) imin = pb[l].ob;
  uint32_t* ring = pm8_ring + threadIdx.x * (RB * CS * W);
  const int top = a.I - 1;
  const int ctop = top / CS, cbot = imin / CS;
  auto issue = [&](int c) {
    if (c >= cbot) {
      uint32_t* slot = ring + (c % RB) * (CS * W);
#pragma unroll
      for (int k = 0; k < CS; ++k) {
        const int i = c * CS + k;
        if (i <= top) {
          const uint32_t* src = a.surv + ((int64_t)i * a.nquads + q) * W;
          const uint32_t d = (uint32_t)__cvta_generic_to_shared(slot + k * W);
          if constexpr (W % 4 == 0) {
#pragma unroll
            for (int w = 0; w < W; w += 4)
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 4 * w), "l"(src + w));
          } else {
#pragma unroll
            for (int w = 0; w < W; w += 2)
              asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 4 * w), "l"(src + w));
          }
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int k = 0; k < RB - 1; ++k) issue(ctop - k);
  int st[4] = {0, 0, 0, 0};
  uint32_t acc[4] = {0, 0, 0, 0};
  for (int c = ctop; c >= cbot; --c) {
    issue(c - (RB - 1));
    asm volatile("cp.async.wait_group %0;" ::"n"(RB - 1) : "memory");
    const uint32_t* slot = ring + (c % RB) * (CS * W);
    const int ihi = top < c * CS + CS - 1 ? top : c * CS + CS - 1;
    const int ilo = imin > c * CS ? imin : c * CS;
    for (int i = ihi; i >= ilo; --i) {
      const uint32_t* rec = slot + (i - c * CS) * W;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        if (i < pb[l].len) {
          if (i >= pb[l].ob && i < pb[l].oe) {
            const int64_t S = pb[l].f0 + i;
            acc[l] |= (uint32_t)((st[l] >> (v - 1)) & 1) << (S & 7);
            if ((S & 7) == 0) {
              a.out[S >> 3] = (uint8_t)acc[l];
              acc[l] = 0;
            }
          }
          const uint32_t up = (rec[st[l] >> 3] >> (8 * l + (st[l] & 7))) & 1u;
          st[l] = ((st[l] & (H - 1)) << 1) | (int)(up ^ 1u);
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Two lanes per quad (64-state codes): lane h holds the states h N/2 ..
// h N/2 + N/2 - 1 of the four blocks (local index k = state - h N/2).  Lane
// h's butterfly jl (jl < N/4) joins its local predecessors 2 jl, 2 jl + 1
// (the states 2 j', 2 j' + 1 with j' = jl + h N/4) into the successors j'
// (lower, lane 0's local j') and j' + N/2 (upper, lane 1's local j'): lane 0
// keeps its lower successors and hands the upper ones to lane 1, lane 1 keeps
// its upper successors and hands the lower ones to lane 0, one shfl.xor per
// butterfly.  Lane 1's codewords are lane 0's xor the taps of the top state
// bit, so each lane relabels its 2^R branch metrics once per stage and the
// butterfly code is the same in both lanes.  The traceback splits the four
// chains over the two lanes.
template <class C, int RKS>
__global__ void __launch_bounds__(32) pm8_decode2_kernel(const Pm8Args a) {
  constexpr int v = C::v, N = C::N, H = C::H, R = C::R, W = C::W;
  constexpr int NL = N / 2, NB = N / 4;  // states and butterflies per lane
  constexpr int NCW = 1 << R;
  constexpr int CS = 8, RB = 4;
  constexpr uint32_t TOP = C::cw(NL, 0);  // codeword taps of state bit v - 1
  static_assert(v % RKS == 0, "renormalisation interval divides the period");
  static_assert(NB % 8 == 0, "whole survivor words per lane");
  extern __shared__ __align__(16) uint32_t pm8_ring[];
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q = gt >> 1;
  const int h = (int)(gt & 1);
  if (q >= a.nquads) return;  // both lanes of a quad leave together
  const unsigned pmask = 3u << (threadIdx.x & 30);
  const uint32_t hm = h ? 0xFFFFFFFFu : 0u;
  Pm8Pb pb[4];
  uint32_t kmask = 0;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    pb[l] = pm8_pb(a, 4 * q + l);
    if (pb[l].len > 0 && pb[l].f0 == 0) kmask |= 0xFFu << (8 * l);
  }
  uint32_t pm[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) pm[k] = a.big4 & kmask;
  pm[0] &= hm;  // S_0 (lane 0, local 0) starts at 0

  const int64_t in_stride = a.nquads * R, sv_stride = a.nquads * W;
  const uint32_t* inp = a.in + q * R;
  uint32_t* svp = a.surv + q * W;
  int per = 0;
  for (int i0 = 0; i0 < a.I; i0 += v) {
    uint32_t x[v][R];
#pragma unroll
    for (int p = 0; p < v; ++p)
#pragma unroll
      for (int r = 0; r < R; ++r) x[p][r] = (i0 + p < a.I) ? __ldg(inp + (int64_t)(i0 + p) * in_stride + r) : 0u;
#pragma unroll
    for (int p = 0; p < v; ++p) {
      if (i0 + p >= a.I) break;
      uint32_t cmp[R], bm[NCW], bl[NCW];
#pragma unroll
      for (int r = 0; r < R; ++r) cmp[r] = a.twoq4 - x[p][r];
#pragma unroll
      for (int c = 0; c < NCW; ++c) {
        uint32_t t = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) t += ((c >> (R - 1 - r)) & 1) ? x[p][r] : cmp[r];
        bm[c] = t;
      }
#pragma unroll
      for (int c = 0; c < NCW; ++c) bl[c] = h ? bm[c ^ TOP] : bm[c];
      uint32_t nw[NL], mlo[NB], mhi[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const uint32_t u0 = pm[2 * j], u1 = pm[2 * j + 1];
        uint32_t o[2];
#pragma unroll
        for (int xb = 0; xb < 2; ++xb) {
          const uint32_t c0 = u0 + bl[C::cw(2 * j, xb)];
          const uint32_t c1 = u1 + bl[C::cw(2 * j + 1, xb)];
          const uint32_t m = sign_mask(c1 + kByteSign - c0);
          o[xb] = (c0 & m) | (c1 & ~m);
          if (xb) mhi[j] = m; else mlo[j] = m;
        }
        const uint32_t send = (o[0] & hm) | (o[1] & ~hm);
        const uint32_t got = __shfl_xor_sync(pmask, send, 1);
        nw[j] = (got & hm) | (o[0] & ~hm);
        nw[j + NB] = (o[1] & hm) | (got & ~hm);
      }
      if (i0 == 0 && kmask) {
#pragma unroll
        for (int k = 0; k < NL; ++k)
          if (k & ((1 << (v - p - 1)) - 1)) nw[k] = (nw[k] & ~kmask) | (a.big4 & kmask);
      }
      uint32_t rl[NB / 8], rh[NB / 8];
#pragma unroll
      for (int w = 0; w < NB / 8; ++w) {
        rl[w] = merge_masks<0, 8>(mlo + 8 * w);
        rh[w] = merge_masks<0, 8>(mhi + 8 * w);
      }
      // lower successors h N/4 + jl: words h NB/8 ..; upper: (H + h NB)/8 ..
      uint32_t* dst = svp + (int64_t)(i0 + p) * sv_stride;
#pragma unroll
      for (int w = 0; w < NB / 8; w += 2) {
        *reinterpret_cast<uint2*>(dst + h * (NB / 8) + w) = make_uint2(rl[w], rl[w + 1]);
        *reinterpret_cast<uint2*>(dst + (H + h * NB) / 8 + w) = make_uint2(rh[w], rh[w + 1]);
      }
#pragma unroll
      for (int k = 0; k < NL; ++k) pm[k] = nw[k];
      bool rn;
      if constexpr (RKS < v) {
        rn = (p + 1) % RKS == 0;
      } else {
        rn = false;
        if (p == v - 1 && ++per == a.rp) {
          per = 0;
          rn = true;
        }
      }
      if (rn) {
        uint32_t t[NL / 2];
#pragma unroll
        for (int j = 0; j < NL / 2; ++j) t[j] = byte_min(pm[2 * j], pm[2 * j + 1]);
#pragma unroll
        for (int w = NL / 4; w >= 1; w /= 2)
#pragma unroll
          for (int j = 0; j < w; ++j) t[j] = byte_min(t[2 * j], t[2 * j + 1]);
        const uint32_t mn = byte_min(t[0], __shfl_xor_sync(pmask, t[0], 1));
#pragma unroll
        for (int k = 0; k < NL; ++k) pm[k] -= mn;
      }
    }
  }

  // traceback: lane h walks the chains of blocks 2h and 2h + 1
  Pm8Pb cb[2];
  cb[0] = h ? pb[2] : pb[0];
  cb[1] = h ? pb[3] : pb[1];
  int imin = a.I;
#pragma unroll
  for (int c = 0; c < 2; ++c)
    if (cb[c].len > 0 && cb[c].ob < imin) imin = cb[c].ob;
  if (imin >= a.I) return;  // neither block exists
  uint32_t* ring = pm8_ring + threadIdx.x * (RB * CS * W);
  const int top = a.I - 1;
  const int ctop = top / CS, cbot = imin / CS;
  auto issue = [&](int c) {
    if (c >= cbot) {
      uint32_t* slot = ring + (c % RB) * (CS * W);
#pragma unroll
      for (int k = 0; k < CS; ++k) {
        const int i = c * CS + k;
        if (i <= top) {
          const uint32_t* src = a.surv + ((int64_t)i * a.nquads + q) * W;
          const uint32_t d = (uint32_t)__cvta_generic_to_shared(slot + k * W);
#pragma unroll
          for (int w = 0; w < W; w += 4)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 4 * w), "l"(src + w));
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int k = 0; k < RB - 1; ++k) issue(ctop - k);
  int st[2] = {0, 0};
  uint32_t acc[2] = {0, 0};
  const int sh0 = 16 * h;  // bit offset of block 2h in a record word
  for (int c = ctop; c >= cbot; --c) {
    issue(c - (RB - 1));
    asm volatile("cp.async.wait_group %0;" ::"n"(RB - 1) : "memory");
    const uint32_t* slot = ring + (c % RB) * (CS * W);
    const int ihi = top < c * CS + CS - 1 ? top : c * CS + CS - 1;
    const int ilo = imin > c * CS ? imin : c * CS;
    for (int i = ihi; i >= ilo; --i) {
      const uint32_t* rec = slot + (i - c * CS) * W;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        if (i < cb[cc].len) {
          if (i >= cb[cc].ob && i < cb[cc].oe) {
            const int64_t S = cb[cc].f0 + i;
            acc[cc] |= (uint32_t)((st[cc] >> (v - 1)) & 1) << (S & 7);
            if ((S & 7) == 0) {
              a.out[S >> 3] = (uint8_t)acc[cc];
              acc[cc] = 0;
            }
          }
          const uint32_t up = (rec[st[cc] >> 3] >> (sh0 + 8 * cc + (st[cc] & 7))) & 1u;
          st[cc] = ((st[cc] & (H - 1)) << 1) | (int)(up ^ 1u);
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <class C, int RKS>
cudaError_t pm8_run2(const Pm8Args& a, cudaStream_t s) {
  constexpr int cta = 32;
  const int64_t grid = (2 * a.nquads + cta - 1) / cta;
  const size_t smem = (size_t)cta * 4 * 8 * C::W * sizeof(uint32_t);
  pm8_decode2_kernel<C, RKS><<<(unsigned)grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C, int RKS>
cudaError_t pm8_run(const Pm8Args& a, cudaStream_t s) {
  constexpr int cta = 32;
  const int64_t grid = (a.nquads + cta - 1) / cta;
  const size_t smem = (size_t)cta * 4 * 8 * C::W * sizeof(uint32_t);
  pm8_decode_kernel<C, RKS><<<(unsigned)grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

using P7 = Pm8Code<7, 0171u, 0133u, 0u>;
using P7R3 = Pm8Code<7, 0171u, 0165u, 0133u>;
using P5 = Pm8Code<5, 023u, 035u, 0u>;

struct Pm8Inst {
  int K, R;
  uint32_t g[3];
  int rks;
  int lanes;  // threads per quad
  cudaError_t (*run)(const Pm8Args&, cudaStream_t);
};

const Pm8Inst kPm8[] = {
    {7, 2, {0171u, 0133u, 0u}, 3, 1, &pm8_run<P7, 3>},
    {7, 2, {0171u, 0133u, 0u}, 6, 1, &pm8_run<P7, 6>},
    {7, 2, {0171u, 0133u, 0u}, 3, 2, &pm8_run2<P7, 3>},
    {7, 2, {0171u, 0133u, 0u}, 6, 2, &pm8_run2<P7, 6>},
    {7, 3, {0171u, 0165u, 0133u}, 1, 1, &pm8_run<P7R3, 1>},
    {7, 3, {0171u, 0165u, 0133u}, 6, 1, &pm8_run<P7R3, 6>},
    {7, 3, {0171u, 0165u, 0133u}, 1, 2, &pm8_run2<P7R3, 1>},
    {7, 3, {0171u, 0165u, 0133u}, 6, 2, &pm8_run2<P7R3, 6>},
    {5, 2, {023u, 035u, 0u}, 4, 1, &pm8_run<P5, 4>},
};

}  // namespace

int pm8_plan(int K, int R, const uint32_t* gens, int q, int lanes, Pm8Plan* p) {
  if (q < 1 || q > 8) return -1;
  const int Q = q == 1 ? 1 : (1 << (q - 1)) - 1;
  const int bmmax = 2 * Q * R;
  if (K * bmmax >= 127) return -1;
  const int k = (127 - K * bmmax) / bmmax + 1;  // candidates stay <= (k - 1 + K) * bmmax <= 127
  const int v = K - 1;
  int best = -1;
  for (int i = 0; i < (int)(sizeof(kPm8) / sizeof(kPm8[0])); ++i) {
    const Pm8Inst& e = kPm8[i];
    if (e.K != K || e.R != R) continue;
    bool same = true;
    for (int r = 0; r < R; ++r) same = same && e.g[r] == gens[r];
    if (!same) continue;
    const bool fits = e.rks < v ? e.rks <= k : k >= v;
    if (!fits || (lanes > 0 && e.lanes != lanes)) continue;
    // the longest renormalisation interval, then the most lanes
    if (best < 0 || e.rks > kPm8[best].rks || (e.rks == kPm8[best].rks && e.lanes > kPm8[best].lanes)) best = i;
  }
  if (best < 0) return -1;
  p->inst = best;
  p->q = q;
  p->Q = Q;
  p->bmmax = bmmax;
  p->rks = kPm8[best].rks;
  p->rp = kPm8[best].rks == v ? k / v : 1;
  p->lanes = kPm8[best].lanes;
  return 0;
}

void pm8_sizes(int K, int R, int64_t n, int D, int L, int64_t* I, int64_t* nquads, size_t* in_words,
               size_t* surv_words) {
  const int64_t nb = (n + D - 1) / D;
  const int64_t span = (int64_t)D + 2 * (int64_t)L;
  *I = span < n ? span : n;
  *nquads = (nb + 3) / 4;
  *in_words = (size_t)(*I) * (size_t)(*nquads) * (size_t)R;
  *surv_words = (size_t)(*I) * (size_t)(*nquads) * (size_t)((1 << (K - 1)) / 8);
}

cudaError_t pm8_launch(const Pm8Plan& p, int K, int R, const uint32_t* words, int64_t n, int D, int L,
                       uint32_t* in, uint32_t* surv, uint8_t* out, cudaStream_t s) {
  Pm8Args a;
  int64_t I, nquads;
  size_t iw, sw;
  pm8_sizes(K, R, n, D, L, &I, &nquads, &iw, &sw);
  a.in = in;
  a.surv = surv;
  a.out = out;
  a.n = n;
  a.nb = (n + D - 1) / D;
  a.nquads = nquads;
  a.D = D;
  a.L = L;
  a.I = (int)I;
  a.rp = p.rp;
  a.big4 = (uint32_t)(127 - p.bmmax) * 0x01010101u;
  a.twoq4 = (uint32_t)(2 * p.Q) * 0x01010101u;
  const dim3 ggrid((unsigned)((nquads + 255) / 256), (unsigned)((I + 31) / 32));
  switch (p.q) {
    case 1: pm8_gather_kernel<1><<<ggrid, 256, 0, s>>>(words, a, R, in); break;
    case 2: pm8_gather_kernel<2><<<ggrid, 256, 0, s>>>(words, a, R, in); break;
    case 3: pm8_gather_kernel<3><<<ggrid, 256, 0, s>>>(words, a, R, in); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return kPm8[p.inst].run(a, s);
}

}  // namespace pbvd
