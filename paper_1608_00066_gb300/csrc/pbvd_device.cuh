// Device code of the parallel block-based Viterbi decoder (sm_103a).
//
// One kernel runs the whole hot path for a set of parallel blocks (PBs):
// soft-value ingest (with depuncturing), branch metrics computed once per
// distinct codeword (Sec. III-B), the add-compare-select recursion of Eq. (1)
// over [f0, f1] (Sec. III-A), bit-packed survivor records, and the traceback
// from S_0 that emits the block's D bits (Algorithm 1, backward procedure).
//
// Data layout (differs from the paper's two-kernel design, see the design
// notes): two PBs are decoded in lock-step by a group of T threads.  Every
// path metric is a 32-bit register holding the same state of both PBs, PB A
// in the low and PB B in the high 16 bits, so one integer instruction serves
// two ACS operations.  A thread holds M = N/T states.
//
// Register layout.  The v bits of a state are stored at "physical" bit
// positions psi: bits [0, r) are the register index k, bits [r, v) the
// thread index tau within the group (r = v - log2 T).  At phase ph of a
// period the state u sits at psi = rotl_v(u, ph).  Then the two predecessors
// of a butterfly (states 2j and 2j+1) are registers k0 and k0 | (1 << ph) of
// one thread, and the two successors (j and j + N/2) land in exactly those
// two registers, so the butterfly is computed in place.  After r stages the
// thread bits have rotated down to the bottom and a transpose through shared
// memory restores psi = u.  With T = 1 the period is v stages and needs no
// transpose.
//
// Metrics are 16-bit lanes kept in [0, 32767], renormalised every few
// stages to PM - PM(S_0) + v * 254 * R.  PM(S_0) is never more than v * 254 * R
// above the smallest metric and never more than 8192 + v * 254 * R below the
// largest (8192 = known-start offset), so after renormalisation every metric
// lies in [0, 2 v 254 R + 8192] (14288 for K=7 R=2, 20384 for K=9 R=3) and
// grows by at most 254 R per stage; renormalising at least every
// (32767 - 254 R - 2 v 254 R - 8192) / (254 R) stages keeps every candidate
// below 32768 and every difference of two candidates below 32768, so the
// 16-bit (signed-safe) arithmetic is exact.
//
// Decision bit of output register k: t = Y - X + (0x8000 + BM(gamma) -
// BM(alpha)) per lane, i.e. 0x8000 + (c1 - c0); bit 15 of each lane is set
// iff c1 >= c0 (the upper branch is kept).  Survivor words store that bit
// (1 = upper branch), 16 registers per word: bit k & 15 for PB A and
// 16 + (k & 15) for PB B.  The traceback walks directly in psi coordinates.
#pragma once

#ifdef __CUDACC_RTC__
#include "pbvd_rtc_types.h"
#else
#include <cstdint>
#include <cuda_runtime.h>
#endif

#include "pbvd_internal.h"

namespace pbvd {

constexpr uint32_t kSignBias = 0x80008000u;  // 0x8000 in both 16-bit lanes
constexpr uint32_t kBigPM = 8192u;            // known-start metric of S_d, d != 0
constexpr uint32_t kLamMax2 = 0x00FE00FEu;    // 254 in both lanes
constexpr int kRing = 16;                      // traceback prefetch: stages per chunk

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// A compile-time int carried by a type (selects a phase in generic lambdas).
template <int V>
struct IntC {
  static constexpr int value = V;
};

// ------------------------------------------------------------------ code --

// An (R,1,K) code with compile-time generators (bit K-1 = input tap).
template <int K_, uint32_t G1, uint32_t G2, uint32_t G3>
struct Code {
  static constexpr int K = K_;
  static constexpr int v = K_ - 1;
  static constexpr int N = 1 << (K_ - 1);
  static constexpr int R = (G3 != 0u) ? 3 : 2;
  static constexpr int NC = 1 << R;  // distinct codewords per stage
  __host__ __device__ static constexpr uint32_t gen(int r) {
    return r == 0 ? G1 : (r == 1 ? G2 : G3);
  }
  // Taps of all R filters at delay position m (Eq. (2)), c^(1) most significant.
  __host__ __device__ static constexpr uint32_t tap(int m) {
    uint32_t c = 0;
    for (int r = 0; r < R; ++r) c = (c << 1) | ((gen(r) >> m) & 1u);
    return c;
  }
  __host__ __device__ static constexpr uint32_t gK() { return tap(K_ - 1); }
  __host__ __device__ static constexpr uint32_t g0() { return tap(0); }
  // alpha = c(S_d, 0) for an even state d: the memory taps D_1..D_{v-1}
  // (Eq. (3)); beta, gamma, theta follow from Eqs. (4)-(6).
  __host__ __device__ static constexpr uint32_t alpha(uint32_t d) {
    uint32_t a = 0;
    for (int m = 1; m < v; ++m)
      if ((d >> m) & 1u) a ^= tap(m);
    return a;
  }
};

template <int v>
__host__ __device__ constexpr uint32_t rotr_v(uint32_t x, int s) {
  return s == 0 ? x : (((x >> s) | (x << (v - s))) & ((1u << v) - 1u));
}
template <int v>
__host__ __device__ constexpr uint32_t rotl_v(uint32_t x, int s) {
  return s == 0 ? x : (((x << s) | (x >> (v - s))) & ((1u << v) - 1u));
}

// Compile-time shape of a (code, T) instance.
template <class C, int T>
struct Shape {
  static constexpr int t = ilog2(T);
  static constexpr int r = C::v - t;               // register-index bits
  static constexpr int M = 1 << r;                 // states per thread
  static constexpr int P = (T == 1) ? C::v : r;    // stages per period
  static constexpr int NB = M / 2;                 // butterflies per thread per stage
  static constexpr int BPW = NB < 8 ? NB : 8;      // butterflies per survivor word
  static constexpr int LBPW = ilog2(BPW);
  static constexpr int W = NB / BPW;               // survivor words per thread per stage
  static constexpr int RW = T * W;                 // survivor words per stage of a pair
  static constexpr int CH = P * ((32 + P - 1) / P);  // stages per staged soft-value chunk
  static constexpr int BMMAX = 254 * C::R;          // largest branch metric
  static constexpr uint32_t RENORM_BASE = (uint32_t)(C::v * BMMAX) * 0x00010001u;
  static constexpr int RENORM_STAGES = (32767 - BMMAX - 2 * C::v * BMMAX - (int)kBigPM) / BMMAX;
  static constexpr int RENORM_PERIODS = RENORM_STAGES / P;
  static_assert(RENORM_PERIODS >= 1, "renormalisation interval shorter than a period");
  static_assert(r >= 1, "at least two states per thread");
  static_assert(T <= 32, "a group lives in one warp");
};

// Per-group shared memory (words).  Forward pass: transpose buffer and two
// raw chunks of soft values per PB.  Traceback (aliases the forward region):
// per-lane rings of survivor records.  The group stride is padded to T
// (mod 32) words so the transpose stores of the groups of a warp fall in
// distinct banks.
template <class C>
__host__ __device__ constexpr int raw_chunk_bytes(int CH) {
  return ((CH * C::R + 15) / 16 + 1) * 16;
}
// Transposes write each thread's registers contiguously (stride M + 4 words)
// and read them back with 16-byte loads when a thread receives at least four
// consecutive registers from each writer (M / T >= 4); otherwise scalar
// stores in natural state order and vector reads.
template <class C, int T>
__host__ __device__ constexpr bool vector_transpose() {
  return T > 1 && (Shape<C, T>::M / T) >= 4;
}
template <class C, int T>
__host__ __device__ constexpr int transpose_words() {
  return (T > 1) ? ((C::N + 4 * T + 3) & ~3) : 0;
}
template <class C, int T>
__host__ __device__ constexpr int raw_offset_words() { return transpose_words<C, T>(); }
// traceback ring per lane: NBUF chunks of KR records of RW words.  Four-word
// records (the v = 6 codes with T <= 4) are walked a period at a time, so a
// chunk is one period and the ring keeps about 24 records in flight.
template <class C, int T>
__host__ __device__ constexpr bool tb_period_walk() {
  return Shape<C, T>::RW == 4 && C::v == 6;
}
template <class C, int T>
__host__ __device__ constexpr int tb_kr() {
  return tb_period_walk<C, T>() ? Shape<C, T>::P
         : T <= 2 ? ((32 / Shape<C, T>::RW) > 1 ? (32 / Shape<C, T>::RW) : 1)
                  : ((16 / Shape<C, T>::RW) > 1 ? (16 / Shape<C, T>::RW) : 1);
}
template <class C, int T>
__host__ __device__ constexpr int tb_nbuf() {
  return tb_period_walk<C, T>() ? 1 + (24 + Shape<C, T>::P - 1) / Shape<C, T>::P : (T <= 2 ? 4 : 3);
}
template <class C, int T>
__host__ __device__ constexpr int scratch_words_per_group() {
  using S = Shape<C, T>;
  const int fwd = raw_offset_words<C, T>() + (2 * 2 * raw_chunk_bytes<C>(S::CH)) / 4;
  const int ring = T * tb_nbuf<C, T>() * tb_kr<C, T>() * S::RW;
  int m = fwd > ring ? fwd : ring;
  m = (m + 3) & ~3;
  // group stride that keeps the transposes of the groups of a warp in
  // distinct banks
  const int want = vector_transpose<C, T>() ? (T == 2 ? 8 : (T == 4 ? 16 : 4)) : ((T < 4 ? 4 : T) & 31);
  while ((m & 31) != want) m += 4;
  return m;
}
template <class C, int T>
__host__ __device__ constexpr int record_words_per_stage() {
  return Shape<C, T>::RW;
}

// ------------------------------------------------------------- soft input --

// One PB of the pair: where its soft values and output bits live and where
// it sits in the lock-step stage index i (i = L is stage bD for every PB).
struct PbRun {
  const int8_t* src;  // soft value with index vidx(f0)
  uint8_t* dst;       // output byte holding stage o0
  int delta;          // lock-step index of stage f0
  int iend;           // lock-step index of stage f1 (-1: no such PB)
  int len;            // f1 - f0 + 1
  int nout;           // o1 - o0
  int f0mod;          // f0 mod P (punctured)
  int known_start;    // f0 == 0: start from the known encoder state S_0
  int rel;            // reader: value index of the next stage, relative to vidx(f0)
  int col;            // reader: column of the next stage (punctured)
};

// Geometry of PB b (Sec. III-A): decodes [bD, min((b+1)D, n)) from the
// forward range [max(0, bD - L), min(n, (b+1)D + L) - 1].
// CIRC: the instance may meet tail-biting frames (KArgs::circular).
template <int R, bool CIRC = false>
__device__ __forceinline__ PbRun pb_run(const KArgs& a, const int8_t* llr, uint8_t* out, int64_t n,
                                        int64_t b) {
  const int D = a.D, L = a.L;
  const int64_t s = b * D - L, e = (b + 1) * D + L;
  int64_t f0 = s < 0 ? 0 : s;
  int64_t f1 = (e < n ? e : n) - 1;
  const int64_t o0 = b * D;
  const int64_t o1 = (b + 1) * D < n ? (b + 1) * D : n;
  const bool circ = CIRC && a.circular;
  if (circ) {
    // tail-biting frame: the window wraps around the frame, read from a copy
    // that holds stages [-L, n + L) (stage s at index s + L)
    f0 = o0 - L;
    f1 = o1 + L - 1;
  }
  PbRun r;
  r.delta = (int)(L - (o0 - f0));
  r.len = (int)(f1 - f0 + 1);
  r.iend = r.delta + r.len - 1;
  r.nout = (int)(o1 - o0);
  r.known_start = (f0 == 0) && !circ;
  r.dst = out + (o0 >> 3);
  int64_t v0;
  if (circ) {
    r.f0mod = 0;
    v0 = (f0 + L) * R;
  } else if (a.punct_P == 0) {
    r.f0mod = 0;
    v0 = f0 * R;
  } else {
    const int64_t per = f0 / a.punct_P;
    r.f0mod = (int)(f0 - per * a.punct_P);
    v0 = per * a.punct_C + a.punct_pre[r.f0mod];
  }
  r.src = llr + v0;
  r.rel = 0;
  r.col = r.f0mod;
  return r;
}

// Value index of the first value of stage f0 + k relative to that of f0.
template <int R>
__device__ __forceinline__ int rel_value_index(const KArgs& a, int f0mod, int k) {
  if (a.punct_P == 0) return k * R;
  const int x = f0mod + k;
  const int per = x / a.punct_P;
  return per * a.punct_C + a.punct_pre[x - per * a.punct_P] - a.punct_pre[f0mod];
}

// Issues the cp.async copies of chunk c (lock-step stages [c*CH, (c+1)*CH))
// of one PB's soft values into 'buf'; lanes lane, lane + nlanes, ... split
// the 16-byte pieces.  Pieces that would reach outside the caller's buffer
// [llr, llr_end) are copied byte by byte with plain loads.  Returns the
// relative value index held by buf[0].
template <int R, int CH>
__device__ __forceinline__ int stage_raw_chunk(const KArgs& a, const PbRun& g, const int8_t* llr,
                                               const int8_t* llr_end, int c, int8_t* buf, int lane,
                                               int nlanes) {
  const int k_lo = max(0, c * CH - g.delta);
  const int k_hi = min(g.len - 1, c * CH + CH - 1 - g.delta);
  if (g.iend < 0 || k_lo > k_hi) return 0;
  const int v0 = rel_value_index<R>(a, g.f0mod, k_lo);
  const int v1 = rel_value_index<R>(a, g.f0mod, k_hi + 1);
  const uintptr_t lo = reinterpret_cast<uintptr_t>(llr), hi = reinterpret_cast<uintptr_t>(llr_end);
  const uintptr_t first = reinterpret_cast<uintptr_t>(g.src) + (uintptr_t)v0;
  const uintptr_t A0 = first & ~(uintptr_t)15;
  const uintptr_t A1 = reinterpret_cast<uintptr_t>(g.src) + (uintptr_t)v1;
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
  return v0 - (int)(first & 15);
}

// Raw bytes (zero-extended) of the R code bits of the reader's next stage
// from the staged chunk 'buf' (whose byte 0 holds relative value index
// cbase); punctured positions read as 0, the byte of soft value 0.  Advances
// the reader.
template <int R, bool PUNCT>
__device__ __forceinline__ void read_raw(const KArgs& a, PbRun& g, const int8_t* buf, int cbase, uint32_t (&u)[3]) {
  const uint8_t* p = reinterpret_cast<const uint8_t*>(buf) + (g.rel - cbase);
  if constexpr (!PUNCT) {
#pragma unroll
    for (int q = 0; q < R; ++q) u[q] = p[q];
    g.rel += R;
  } else {
    int used = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int off = a.punct_off[g.col * 4 + q];
      u[q] = off >= 0 ? (uint32_t)p[used] : 0u;
      used += off >= 0;
    }
    g.rel += used;
    if (++g.col == a.punct_P) g.col = 0;
  }
}

// 127 + max(lambda, -127) per 16-bit lane from sign-extended soft values:
// max(lambda + 127, 0) in one fused add-max (lambda = -128 gives 0).
__device__ __forceinline__ uint32_t soft_lanes(uint32_t x) {
  return __viaddmax_s16x2_relu(x, 0x007F007Fu, 0u);
}

// Packs the raw soft-value bytes of PB A (low lane) and PB B (high lane):
// byte permute with sign replication (selector nibbles 8 and C copy the sign
// of bytes 0 and 4) into two sign-extended 16-bit lanes, then soft_lanes.
__device__ __forceinline__ uint32_t pack_soft(uint32_t ua, uint32_t ub) {
  uint32_t x;
  asm("prmt.b32 %0, %1, %2, 0xC480;" : "=r"(x) : "r"(ua), "r"(ub));
  return soft_lanes(x);
}

// ------------------------------------------------------------ ACS stage --

// Branch metrics of all 2^R codewords for both PBs of the pair, and the
// decision constants kt[c] = 0x8000 + BM(c ^ g0) - BM(c) per lane.  sel[q]
// is all-ones where this thread relabels code bit q: the butterfly at
// compile-time register k0 belongs to group alpha(k0) ^ swp (see thread_swap).
template <class C, bool SWAP>
__device__ __forceinline__ void branch_metrics(const uint32_t (&Pk)[3], const uint32_t (&sel)[3],
                                               uint32_t (&bm)[C::NC], uint32_t (&kt)[C::NC]) {
  constexpr int R = C::R;
  uint32_t Pp[3], Mp[3];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    // lane value for code bit 1 is 127 + lambda (distance to -127), for bit 0
    // it is 127 - lambda
    const uint32_t m1 = Pk[q], m0 = kLamMax2 - Pk[q];
    if constexpr (SWAP) {
      Pp[q] = (m1 & ~sel[q]) | (m0 & sel[q]);
      Mp[q] = kLamMax2 - Pp[q];
    } else {
      Pp[q] = m1;
      Mp[q] = m0;
    }
  }
  constexpr uint32_t FULL = (uint32_t)C::NC - 1u;
  if constexpr (C::g0() == FULL) {
    // every generator taps the oldest cell, so BM(c ^ g0) = 254 R - BM(c):
    // half the sums, the other half by complement, and kt[c] =
    // 254 R + 0x8000 - 2 BM(c) per lane (no borrow between the lanes)
    constexpr uint32_t SUM = (uint32_t)(254 * R) * 0x00010001u;
#pragma unroll
    for (int c = 0; c < C::NC / 2; ++c) {
      uint32_t s = 0;
#pragma unroll
      for (int q = 0; q < R; ++q) s += ((c >> (R - 1 - q)) & 1) ? Pp[q] : Mp[q];
      bm[c] = s;
      bm[c ^ FULL] = SUM - s;
    }
#pragma unroll
    for (int c = 0; c < C::NC; ++c) kt[c] = (SUM + kSignBias) - 2u * bm[c];
  } else {
#pragma unroll
    for (int c = 0; c < C::NC; ++c) {
      uint32_t s = 0;
#pragma unroll
      for (int q = 0; q < R; ++q) s += ((c >> (R - 1 - q)) & 1) ? Pp[q] : Mp[q];
      bm[c] = s;
    }
#pragma unroll
    for (int c = 0; c < C::NC; ++c) kt[c] = bm[c ^ C::g0()] + kSignBias - bm[c];
  }
}

// Byte masks of the four decisions of a butterfly: bytes 1 and 3 of t0 and
// t1 hold the decisions in their sign bit; prmt with the sign-replicating
// selector nibbles 9, B, D, F turns each into a 0x00 / 0xFF byte.
__device__ __forceinline__ uint32_t decision_bytes(uint32_t t0, uint32_t t1) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, 0xFDB9;" : "=r"(r) : "r"(t0), "r"(t1));
  return r;
}

// Merges the byte masks d[lo..lo+n) of consecutive butterflies into one
// word: butterfly q's decisions end up at bit q of every byte.  The masks
// are all-zero or all-one bytes, so a select with a constant needs no shift.
template <int LO, int N>
__device__ __forceinline__ uint32_t merge_decisions(const uint32_t* d) {
  if constexpr (N == 1) {
    return d[LO];
  } else {
    const uint32_t a = merge_decisions<LO, N / 2>(d);
    const uint32_t b = merge_decisions<LO + N / 2, N / 2>(d);
    constexpr uint32_t byte = ((1u << (N / 2)) - 1u) << (LO + N / 2);
    constexpr uint32_t m = byte * 0x01010101u;
    return (a & ~m) | (b & m);
  }
}

// One trellis stage at phase PH for the thread's M registers, in place.
// Butterfly b (the b-th register k0 with bit PH clear, k1 = k0 | 1 << PH)
// stores its four decision bits in survivor word b / BPW at bits q (PB A of
// k0), 8 + q (PB B of k0), 16 + q (PB A of k1), 24 + q (PB B of k1),
// q = b % BPW; a set bit means the upper branch was kept.
// Per butterfly: two fused 16x2 add-min, two candidate adds, two
// three-input decision differences, one byte permute and 7/8 of a select for
// the decision bits (the compiler spreads the adds over the ALU and FMA
// pipes).
template <class C, int T, int PH>
__device__ __forceinline__ void acs_stage(uint32_t (&pm)[Shape<C, T>::M], uint32_t (&wd)[Shape<C, T>::W],
                                          const uint32_t (&bm)[C::NC], const uint32_t (&kt)[C::NC]) {
  using S = Shape<C, T>;
  constexpr uint32_t g0 = C::g0(), gK = C::gK();
#pragma unroll
  for (int w = 0; w < S::W; ++w) {
    uint32_t d[S::BPW];
#pragma unroll
    for (int q = 0; q < S::BPW; ++q) {
      const int b = w * S::BPW + q;
      const int k0 = ((b >> PH) << (PH + 1)) | (b & ((1 << PH) - 1));
      const int k1 = k0 | (1 << PH);
      const uint32_t al = C::alpha(rotr_v<C::v>((uint32_t)k0, PH));
      const uint32_t be = al ^ gK;
      const uint32_t X = pm[k0], Y = pm[k1];
      const uint32_t c1 = Y + bm[al ^ g0];
      const uint32_t c3 = Y + bm[be ^ g0];
      const uint32_t t0 = Y + kt[al] - X;
      const uint32_t t1 = Y + kt[be] - X;
      pm[k0] = __viaddmin_s16x2(X, bm[al], c1);
      pm[k1] = __viaddmin_s16x2(X, bm[be], c3);
      d[q] = decision_bytes(t0, t1);
    }
    wd[w] = merge_decisions<0, S::BPW>(d);
  }
}

// Codeword relabelling of thread tau at phase ph: the thread bits of the
// physical index contribute alpha(rotr(tau << r, ph)) to every butterfly's
// group (alpha is linear in the state bits).
template <class C, int T>
__device__ __forceinline__ uint32_t thread_swap(int tau, int ph) {
  using S = Shape<C, T>;
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < S::t; ++j)
    if ((tau >> j) & 1) m ^= C::alpha(rotr_v<C::v>(1u << (S::r + j), ph));
  return m;
}

// The state with the smallest metric of PB x (0: low lanes, 1: high lanes)
// over the group's N states, after a stage of phase ph, when state u sits at
// physical index psi = rotl_v(u, ph + 1); ties keep the lowest state index
// (the start state S_E of the classic VA, Sec. II).  Returns its physical
// index, where the traceback of that stage starts.  All T lanes of the group
// must call it together.
template <class C, int T>
__device__ __forceinline__ int argmin_state(const uint32_t (&pm)[Shape<C, T>::M], int tau, unsigned gmask, int ph,
                                            int x) {
  using S = Shape<C, T>;
  const int rot = (ph + 1) % C::v;
  uint32_t best = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < S::M; ++k) {
    const uint32_t m = x ? (pm[k] >> 16) : (pm[k] & 0xffffu);
    const uint32_t u = rotr_v<C::v>(((uint32_t)tau << S::r) | (uint32_t)k, rot);
    const uint32_t key = (m << 9) | u;
    best = key < best ? key : best;
  }
  if constexpr (T > 1) {
#pragma unroll
    for (int off = 1; off < T; off <<= 1) {
      const uint32_t o = __shfl_xor_sync(gmask, best, off, T);
      best = o < best ? o : best;
    }
  }
  return (int)rotl_v<C::v>(best & 0x1ffu, rot);
}

// ------------------------------------------------------------- the kernel --

template <class C, int T>
__device__ __forceinline__ void reinit_lane(uint32_t (&pm)[Shape<C, T>::M], int tau, uint32_t lane_mask,
                                            bool known_start) {
  using S = Shape<C, T>;
#pragma unroll
  for (int k = 0; k < S::M; ++k) {
    const uint32_t init = known_start ? ((tau == 0 && k == 0) ? 0u : (kBigPM | (kBigPM << 16))) : 0u;
    pm[k] = (pm[k] & ~lane_mask) | (init & lane_mask);
  }
}

// Source of one PB: its stream (soft values, output bytes, length) and its
// index in that stream.
struct PbSrc {
  const int8_t* llr;
  const int8_t* llr_end;  // end of the readable soft values
  uint8_t* out;
  int64_t n;              // stages of the stream
  int64_t b;              // block index within the stream
};

// Work item of one group: a pair of PBs, possibly of different streams.
struct PairWork {
  PbSrc A, B;
  bool hasB;              // second PB exists
};

// One period (P stages starting at lock-step index i0) of the forward pass.
// CHECKED = false: every stage of the period is inside both PBs' forward
// ranges (or B does not exist) and no re-initialisation falls inside; then
// STORE says whether all of its stages (i >= L) or none of them keep
// survivor records, so the period is one branch-free basic block.  SMEM:
// records go to shared memory (ssv), else to the global workspace (gsv).
template <class C, int T, bool CHECKED, bool PUNCT, bool SMEM, bool STORE, bool CAP = false>
__device__ __forceinline__ void forward_period(uint32_t (&pm)[Shape<C, T>::M], const uint32_t (&sel)[Shape<C, T>::P][3],
                                               const KArgs& a, const int8_t* bufA, int cbA, const int8_t* bufB,
                                               int cbB, bool hasB, int i0, int I, int L, int tau, PbRun& gA,
                                               PbRun& gB, uint32_t*& gsv, int64_t rec_stride, uint32_t*& ssv,
                                               int* start = nullptr, unsigned gmask = 0u) {
  using S = Shape<C, T>;
  constexpr int W = S::W;
  constexpr int R = C::R;
  // the soft values of the whole period, read and packed up front
  uint32_t pkv[S::P][3];
  if constexpr (!CHECKED && !PUNCT && R == 2) {
    // both code bits of a stage in one 2-byte load (even offsets)
    const uint16_t* pa = reinterpret_cast<const uint16_t*>(bufA + (gA.rel - cbA));
    const uint16_t* pb = reinterpret_cast<const uint16_t*>(bufB + (gB.rel - cbB));
#pragma unroll
    for (int ph = 0; ph < S::P; ++ph) {
      const uint32_t wa = pa[ph], wb = pb[ph];
      uint32_t x0, x1;
      asm("prmt.b32 %0, %1, %2, 0xC480;" : "=r"(x0) : "r"(wa), "r"(wb));
      asm("prmt.b32 %0, %1, %2, 0xD591;" : "=r"(x1) : "r"(wa), "r"(wb));
      pkv[ph][0] = soft_lanes(x0);
      pkv[ph][1] = soft_lanes(x1);
      pkv[ph][2] = 0u;
    }
    gA.rel += 2 * S::P;
    gB.rel += 2 * S::P;
  } else {
#pragma unroll
    for (int ph = 0; ph < S::P; ++ph) {
      const int i = i0 + ph;
      uint32_t ua[3] = {0u, 0u, 0u}, ub[3] = {0u, 0u, 0u};
      const bool va = !CHECKED || (i < I && i >= gA.delta && i <= gA.iend);
      const bool vb = hasB && (!CHECKED || (i < I && i >= gB.delta && i <= gB.iend));
      if (va) read_raw<R, PUNCT>(a, gA, bufA, cbA, ua);
      if (vb) read_raw<R, PUNCT>(a, gB, bufB, cbB, ub);
#pragma unroll
      for (int q = 0; q < 3; ++q) pkv[ph][q] = q < R ? pack_soft(ua[q], ub[q]) : 0u;
    }
  }
#pragma unroll
  for (int ph = 0; ph < S::P; ++ph) {
    const int i = i0 + ph;
    if (CHECKED) {
      if (i >= I) break;
      if (i == gA.delta && i != 0) reinit_lane<C, T>(pm, tau, 0x0000ffffu, gA.known_start);
      if (i == gB.delta && i != 0) reinit_lane<C, T>(pm, tau, 0xffff0000u, gB.known_start);
    }
    const uint32_t (&Pk)[3] = pkv[ph];
    uint32_t bm[C::NC], kt[C::NC];
    branch_metrics<C, (T > 1)>(Pk, sel[ph], bm, kt);
    uint32_t wd[W];
    // ph is a compile-time constant after unrolling
    if constexpr (S::P > 0) if (ph == 0) acs_stage<C, T, 0>(pm, wd, bm, kt);
    if constexpr (S::P > 1) if (ph == 1) acs_stage<C, T, (S::P > 1 ? 1 : 0)>(pm, wd, bm, kt);
    if constexpr (S::P > 2) if (ph == 2) acs_stage<C, T, (S::P > 2 ? 2 : 0)>(pm, wd, bm, kt);
    if constexpr (S::P > 3) if (ph == 3) acs_stage<C, T, (S::P > 3 ? 3 : 0)>(pm, wd, bm, kt);
    if constexpr (S::P > 4) if (ph == 4) acs_stage<C, T, (S::P > 4 ? 4 : 0)>(pm, wd, bm, kt);
    if constexpr (S::P > 5) if (ph == 5) acs_stage<C, T, (S::P > 5 ? 5 : 0)>(pm, wd, bm, kt);
    if constexpr (S::P > 6) if (ph == 6) acs_stage<C, T, (S::P > 6 ? 6 : 0)>(pm, wd, bm, kt);
    if constexpr (S::P > 7) if (ph == 7) acs_stage<C, T, (S::P > 7 ? 7 : 0)>(pm, wd, bm, kt);
    if constexpr (CAP && CHECKED) {
      // argmin traceback start: the metrics right after each PB's last stage
      if (a.tb_argmin) {
        if (i == gA.iend) start[0] = argmin_state<C, T>(pm, tau, gmask, ph, 0);
        if (hasB && i == gB.iend) start[1] = argmin_state<C, T>(pm, tau, gmask, ph, 1);
      }
    }
    if (CHECKED ? (i >= L) : STORE) {
      if constexpr (SMEM) {
#pragma unroll
        for (int w = 0; w < W; ++w) ssv[w] = wd[w];
        ssv += S::RW;
      } else {
        uint32_t* d = gsv;
        if constexpr (W % 4 == 0) {
#pragma unroll
          for (int w = 0; w < W; w += 4)
            *reinterpret_cast<uint4*>(d + w) = make_uint4(wd[w], wd[w + 1], wd[w + 2], wd[w + 3]);
        } else if constexpr (W == 2) {
          *reinterpret_cast<uint2*>(d) = make_uint2(wd[0], wd[1]);
        } else {
          d[0] = wd[0];
        }
        gsv += rec_stride;
      }
    }
  }
}

// ------------------------------------------------------------- traceback --

// Traceback shape.  Every lane walks both PBs of its pair (two chains over
// the same records).  T == 1: all records, from S_0.  T >= 2: the records
// are split into T segments of whole bytes, lane tau walking segment tau;
// each non-top segment starts LAMBDA records above its range from S_0 (a
// guess), then is checked against the exact exit state of the segment above
// and re-walked if it differs, so the result is exact for any LAMBDA.
template <class C, int T>
struct TbShape {
  static constexpr int RW = Shape<C, T>::RW;             // words per record
  static constexpr int KR = tb_kr<C, T>();                // records per prefetch chunk
  static constexpr int NBUF = tb_nbuf<C, T>();            // chunks in the per-lane ring
  static constexpr int RING_WORDS = NBUF * KR * RW;       // per lane
  static constexpr int LAMBDA = 8 * C::K;                 // warm-up records of a guessed segment
};

// One traceback step at a stage record rec (shared memory) for the state at
// physical index psi; lm = (1 << ph) - 1 for the stage's phase ph.  In psi
// coordinates the decoded bit is bit ph of psi and the predecessor replaces
// that bit by the survivor bit; after phase 0 the index rotates into the
// layout of the period before.  Returns the decoded bit.
template <class C, int T>
__device__ __forceinline__ int tb_step(int& psi, int& lm, int x, const uint32_t* rec) {
  using S = Shape<C, T>;
  constexpr int P = S::P;
  constexpr int LMTOP = (1 << (P - 1)) - 1;
  const int k = psi & (S::M - 1);
  const int phb = lm + 1;
  const int h = (k & phb) ? 1 : 0;
  const int b = ((k >> 1) & ~lm) | (k & lm);
  const int wi = (psi >> S::r) * S::W + (b >> S::LBPW);
  const int bitpos = (((h << 1) | x) << 3) + (b & (S::BPW - 1));
  const int upper = (rec[wi] >> bitpos) & 1;
  const int np = (psi & ~phb) | (upper ? 0 : phb);
  const bool wrap = (lm == 0);
  psi = wrap ? (int)rotl_v<C::v>((uint32_t)np, P % C::v) : np;
  lm = wrap ? LMTOP : (lm >> 1);
  return h;
}

// tb_step on a four-word record held in registers (RW == 4): the record can
// be loaded before the state that indexes it is known, so the shared-memory
// load leaves the step's dependency chain.
template <class C, int T>
__device__ __forceinline__ int tb_step4(int& psi, int& lm, int x, const uint4& rec) {
  using S = Shape<C, T>;
  static_assert(S::RW == 4, "four-word records");
  constexpr int P = S::P;
  constexpr int LMTOP = (1 << (P - 1)) - 1;
  const int k = psi & (S::M - 1);
  const int phb = lm + 1;
  const int h = (k & phb) ? 1 : 0;
  const int b = ((k >> 1) & ~lm) | (k & lm);
  const int wi = (psi >> S::r) * S::W + (b >> S::LBPW);
  const int bitpos = (((h << 1) | x) << 3) + (b & (S::BPW - 1));
  const uint32_t lo = (wi & 1) ? rec.y : rec.x;
  const uint32_t hi = (wi & 1) ? rec.w : rec.z;
  const uint32_t word = (wi & 2) ? hi : lo;
  const int upper = (word >> bitpos) & 1;
  const int np = (psi & ~phb) | (upper ? 0 : phb);
  const bool wrap = (lm == 0);
  psi = wrap ? (int)rotl_v<C::v>((uint32_t)np, P % C::v) : np;
  lm = wrap ? LMTOP : (lm >> 1);
  return h;
}

// Global address of survivor record j of the group.
template <class C, int T>
__device__ __forceinline__ const uint32_t* global_record(const KArgs& a, int64_t gslot, int j) {
  return a.surv + ((int64_t)j * a.surv_pairs + gslot) * a.surv_rs;
}

// Walks records [lo, hs] of NCH chains (descending) and emits, for records
// j <= emit_top[c], bit (j & 7) of output byte j >> 3 (bits of stages at or
// beyond nout are cleared).  Records are read from shared memory: the
// survivor region svs in shared-memory mode, else a per-lane ring that is
// filled with cp.async KR records at a time.  On return psi is the exit
// state and g the state held on arrival at record g_at.
template <class C, int T, bool SMEM, int NCH>
__device__ __forceinline__ void tb_walk(const KArgs& a, int64_t gslot, const uint32_t* svs, uint32_t* ring,
                                        int L, int hs, int lo, const int (&emit_top)[NCH], const int (&jend)[NCH],
                                        const int (&x)[NCH], const int (&nout)[NCH], uint8_t* const (&dst)[NCH],
                                        int g_at, int (&psi)[NCH], int (&g)[NCH]) {
  using TS = TbShape<C, T>;
  constexpr int P = Shape<C, T>::P, RW = TS::RW, KR = TS::KR, NBUF = TS::NBUF;
  int lm[NCH];
  uint32_t acc[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    lm[c] = (1 << ((L + max(0, min(hs, jend[c]))) % P)) - 1;
    acc[c] = 0u;
    g[c] = 0;
  }
  if (hs < lo) return;
  auto emit = [&](int c, int j, int bit) {
    acc[c] = (acc[c] << 1) | (uint32_t)bit;
    if ((j & 7) == 0 && j <= emit_top[c]) {
      const int rem = nout[c] - j;
      const uint32_t keep = rem >= 8 ? 0xffu : ((1u << (rem > 0 ? rem : 0)) - 1u);
      // the last 8 steps shifted in stages j + 7 .. j: bit q is stage j + q
      dst[c][j >> 3] = (uint8_t)(acc[c] & keep);
    }
  };
  auto visit = [&](int j, const uint32_t* rec) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (j <= jend[c]) {
        g[c] = (j == g_at) ? psi[c] : g[c];
        emit(c, j, tb_step<C, T>(psi[c], lm[c], x[c], rec));
      }
    }
  };
  // four-word records: r[q] = record jtop - q, all loaded before the walk
  // through them (records below jbot are loaded but not visited)
  auto visit4 = [&](int jtop, int jbot, const uint32_t* rec_top, int step) {
    if constexpr (RW == 4) {
      uint4 r[KR];
#pragma unroll
      for (int q = 0; q < KR; ++q) r[q] = *reinterpret_cast<const uint4*>(rec_top + q * step);
#pragma unroll
      for (int q = 0; q < KR; ++q) {
        const int j = jtop - q;
        if (j >= jbot) {
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            if (j <= jend[c]) {
              g[c] = (j == g_at) ? psi[c] : g[c];
              emit(c, j, tb_step4<C, T>(psi[c], lm[c], x[c], r[q]));
            }
          }
        }
      }
    }
  };
  if constexpr (SMEM) {
    if constexpr (RW == 4) {
      for (int jtop = hs; jtop >= lo; jtop -= KR) {
        const int jbot = max(lo, jtop - KR + 1);
        if (jtop - KR + 1 >= 0) {
          visit4(jtop, jbot, svs + jtop * RW, -RW);
        } else {
          for (int j = jtop; j >= jbot; --j) visit(j, svs + j * RW);
        }
      }
    } else {
      for (int j = hs; j >= lo; --j) visit(j, svs + j * RW);
    }
    return;
  }
  // ring: chunk ch holds records hs - ch*KR - q, q < KR, in buffer ch % NBUF
  const int nchunk = (hs - lo) / KR + 1;
  const int64_t stride = a.surv_pairs * (int64_t)a.surv_rs;
  const uint32_t* src_next = global_record<C, T>(a, gslot, hs);
  // ring positions of the next request (iq) and of the next chunk walked
  // (ic), kept running
  int issued = 0, iq = 0, ic = 0;
  auto issue = [&]() {
    if (issued < nchunk) {
      uint32_t* dst0 = ring + iq * (KR * RW);
      const int jtop = hs - issued * KR;
#pragma unroll
      for (int q = 0; q < KR; ++q) {
        if (jtop - q >= lo) {
          const unsigned d = (unsigned)__cvta_generic_to_shared(dst0 + q * RW);
          if constexpr (RW >= 4) {
#pragma unroll
            for (int w = 0; w < RW; w += 4)
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 4 * w), "l"(src_next + w));
          } else if constexpr (RW == 2) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src_next));
          } else {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src_next));
          }
          src_next -= stride;
        }
      }
    }
    ++issued;
    iq = (iq + 1 == NBUF) ? 0 : iq + 1;
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int q = 0; q < NBUF - 1; ++q) issue();
  for (int ch = 0; ch < nchunk; ++ch) {
    issue();
    asm volatile("cp.async.wait_group %0;" ::"n"(NBUF - 1) : "memory");
    const int jtop = hs - ch * KR;
    const int jbot = max(lo, jtop - KR + 1);
    const uint32_t* buf = ring + ic * (KR * RW);
    ic = (ic + 1 == NBUF) ? 0 : ic + 1;
    if constexpr (RW == 4) {
      visit4(jtop, jbot, buf, RW);
    } else {
      for (int j = jtop; j >= jbot; --j) visit(j, buf + (jtop - j) * RW);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}


// ----------------------------------------------- period-unrolled traceback --
//
// For four-word records (v = 6, T * NB = 32 butterflies per stage and PB
// pair) the survivor bit of the state at physical index psi in a record of
// phase ph sits at word B >> 3, byte 2h + x, bit B & 7, where B is psi with
// bit ph deleted (5 bits) and h = bit ph of psi.  gather4 moves the 64 bits
// of PB x into one 64-bit value G whose byte g holds record word g >> 1,
// byte 2 (g & 1) + x, i.e. bit (B4 B3 h B2 B1 B0) of G; at phase 4 the bytes
// are ordered (B4, h, B3) instead.  Then the bit of psi is bit conv4(psi)
// of G, and conv4 is the identity at phases 3 and 4.
template <int PH>
__device__ __forceinline__ uint64_t gather4(const uint4& rec, int x) {
  const uint32_t sel = PH == 4 ? (x ? 0x7351u : 0x6240u) : (x ? 0x7531u : 0x6420u);
  const uint32_t g0 = __byte_perm(rec.x, rec.y, sel);
  const uint32_t g1 = __byte_perm(rec.z, rec.w, sel);
  return ((uint64_t)g1 << 32) | g0;
}

template <int PH>
__device__ __forceinline__ uint32_t conv4(uint32_t psi) {
  if constexpr (PH == 3 || PH == 4) {
    return psi;
  } else if constexpr (PH == 5) {
    // B = (p4 p3 p2 p1 p0), h = p5: bit index (p4 p3 p5 p2 p1 p0)
    return ((psi << 1) & 0x30u) | ((psi >> 2) & 0x8u) | (psi & 0x7u);
  } else {
    // B = (p5 p4 [p3 p2 p1 p0 without p_PH]), h = p_PH
    const uint32_t low = psi & ((1u << PH) - 1u);
    const uint32_t mid = (psi >> (PH + 1)) & ((1u << (3 - PH)) - 1u);
    return (psi & 0x30u) | (((psi >> PH) & 1u) << 3) | (mid << PH) | low;
  }
}

// One traceback step at a record of compile-time phase PH: appends the
// decoded bit (bit PH of psi) to acc (ACC) and moves psi to the predecessor
// (bit PH replaced by the survivor's branch, then the period rotation at
// PH = 0).  Over a whole period (phases P-1 .. 0) step PH reads bit PH
// before any step changes it, so the period's P decoded bits are the low P
// bits of psi on entry; the unguarded walk appends them once per period.
template <class C, int T, int PH, bool ACC = true>
__device__ __forceinline__ void tb_step_ph(uint32_t& psi, uint32_t& acc, uint64_t G) {
  constexpr int P = Shape<C, T>::P;
  const uint32_t upper = (uint32_t)(G >> conv4<PH>(psi)) & 1u;
  if constexpr (ACC) acc = (acc << 1) | ((psi >> PH) & 1u);
  uint32_t np = (psi & ~(1u << PH)) | ((upper ^ 1u) << PH);
  if constexpr (PH == 0) np = rotl_v<C::v>(np, P % C::v);
  psi = np;
}

// tb_walk for four-word records: the records [lo, hs] are visited in blocks
// of one period (phases P-1 .. 0, so every step has a compile-time phase);
// blocks wholly inside every chain's range and not holding g_at run without
// per-record guards.  A block's records come from the shared-memory
// survivors or from a ring of NBUF blocks filled with cp.async.  Output bytes
// are written once per block from the bit accumulator.
template <class C, int T, bool SMEM, int NCH>
__device__ __forceinline__ void tb_walk4(const KArgs& a, int64_t gslot, const uint32_t* svs, uint32_t* ring,
                                         int L, int hs, int lo, const int (&emit_top)[NCH],
                                         const int (&jend)[NCH], const int (&x)[NCH], const int (&nout)[NCH],
                                         uint8_t* const (&dst)[NCH], int g_at, int (&psi)[NCH], int (&g)[NCH]) {
  constexpr int P = Shape<C, T>::P, NBUF = tb_nbuf<C, T>();
  static_assert(tb_kr<C, T>() == P, "one period per ring chunk");
  uint32_t ps[NCH], acc[NCH];
  int jmax = jend[0];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    ps[c] = (uint32_t)psi[c];
    acc[c] = 0u;
    g[c] = 0;
    jmax = min(jmax, jend[c]);
  }
  if (hs < lo) return;
  // block k holds records atop - k P - u, u = 0..P-1, at phases P-1-u
  const int atop = hs + (P - 1 - (L + hs) % P);
  const int nblk = (atop - lo) / P + 1;
  // Global mode: the next block to request starts at record jq, whose word
  // offset in the workspace is offq; consecutive records of a slot lie
  // 'stride' words apart, so the offsets are kept running (no per-record
  // multiply) and so are the ring positions of the next request (iq) and of
  // the next block walked (ic).
  const int64_t stride = a.surv_pairs * (int64_t)a.surv_rs;
  int64_t offq = ((int64_t)atop * a.surv_pairs + gslot) * a.surv_rs;
  int jq = atop;
  int iq = 0, ic = 0;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  auto issue = [&]() {
    if constexpr (!SMEM) {
      if (jq >= lo) {
        const unsigned d0 = ring_s + (unsigned)iq * (P * 16);
        const uint32_t* src = a.surv + offq;
        if (jq <= hs && jq - (P - 1) >= lo) {
#pragma unroll
          for (int u = 0; u < P; ++u) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16 * u), "l"(src));
            src -= stride;
          }
        } else {
#pragma unroll
          for (int u = 0; u < P; ++u) {
            const int j = jq - u;
            if (j >= lo && j <= hs)
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16 * u), "l"(src));
            src -= stride;
          }
        }
      }
      offq -= P * stride;
      jq -= P;
      iq = (iq + 1 == NBUF) ? 0 : iq + 1;
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  };
#pragma unroll
  for (int q = 0; q < NBUF - 1; ++q) issue();
  for (int k = 0; k < nblk; ++k) {
    const int j0 = atop - k * P;
    const uint32_t* blk;
    int bstep;
    if constexpr (SMEM) {
      blk = svs + (int64_t)j0 * 4;
      bstep = -4;
    } else {
      issue();
      asm volatile("cp.async.wait_group %0;" ::"n"(NBUF - 1) : "memory");
      blk = ring + ic * (P * 4);
      ic = (ic + 1 == NBUF) ? 0 : ic + 1;
      bstep = 4;
    }
    const int jb = max(lo, j0 - P + 1);
    const bool full = j0 <= hs && j0 - P + 1 >= lo && j0 <= jmax && (g_at > j0 || g_at < j0 - P + 1);
    uint4 rec[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
      // a ring slot always lies inside the lane's ring (records outside
      // [lo, hs] are loaded but never walked); the shared-memory survivor
      // region is read only inside the group's records
      const int j = j0 - u;
      if (!SMEM || full || (j >= lo && j <= hs)) rec[u] = *reinterpret_cast<const uint4*>(blk + u * bstep);
    }
    auto step = [&](auto phc, int u, auto guarded) {
      constexpr int PH = decltype(phc)::value;
      constexpr bool G = decltype(guarded)::value != 0;
      const int j = j0 - u;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        if (!G || (j >= lo && j <= hs && j <= jend[c])) {
          if (G && j == g_at) g[c] = (int)ps[c];
          tb_step_ph<C, T, PH, G>(ps[c], acc[c], gather4<PH>(rec[u], x[c]));
        }
      }
    };
    auto run_block = [&](auto guarded) {
      if constexpr (decltype(guarded)::value == 0) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) acc[c] = (acc[c] << P) | (ps[c] & ((1u << P) - 1u));
      }
      if constexpr (P > 5) step(IntC<(P > 5 ? P - 6 : 0) + 5>{}, P - 6, guarded);
      if constexpr (P > 4) step(IntC<4>{}, P - 5, guarded);
      step(IntC<3>{}, P - 4, guarded);
      step(IntC<2>{}, P - 3, guarded);
      step(IntC<1>{}, P - 2, guarded);
      step(IntC<0>{}, P - 1, guarded);
    };
    if (full) run_block(IntC<0>{}); else run_block(IntC<1>{});
    // the byte whose lowest record (a multiple of 8) lies in this block
    const int m8 = (j0 >> 3) << 3;
    if (m8 >= jb && m8 <= hs) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        if (m8 <= emit_top[c] && m8 <= jend[c]) {
          const int rem = nout[c] - m8;
          const uint32_t keep = rem >= 8 ? 0xffu : ((1u << (rem > 0 ? rem : 0)) - 1u);
          dst[c][m8 >> 3] = (uint8_t)((acc[c] >> (m8 - jb)) & keep);
        }
      }
    }
  }
  if constexpr (!SMEM) asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
  for (int c = 0; c < NCH; ++c) psi[c] = (int)ps[c];
}

template <class C, int T, bool SMEM, int NCH>
__device__ __forceinline__ void tb_walk_any(const KArgs& a, int64_t gslot, const uint32_t* svs, uint32_t* ring,
                                            int L, int hs, int lo, const int (&emit_top)[NCH],
                                            const int (&jend)[NCH], const int (&x)[NCH], const int (&nout)[NCH],
                                            uint8_t* const (&dst)[NCH], int g_at, int (&psi)[NCH], int (&g)[NCH]) {
  if constexpr (tb_period_walk<C, T>())
    tb_walk4<C, T, SMEM, NCH>(a, gslot, svs, ring, L, hs, lo, emit_top, jend, x, nout, dst, g_at, psi, g);
  else
    tb_walk<C, T, SMEM, NCH>(a, gslot, svs, ring, L, hs, lo, emit_top, jend, x, nout, dst, g_at, psi, g);
}

// start[x]: physical index of the state PB x's traceback starts from at its
// last forward stage (0 = S_0, whose index is 0 in every layout).  PAR: walk
// failed guesses again side by side before the top-down check (the batch
// kernels leave it out: in their register budget it costs spills).
template <class C, int T, bool SMEM, bool PAR = true>
__device__ __forceinline__ void traceback_pair(const KArgs& a, const PbRun& gA, const PbRun& gB, bool hasB, int J,
                                               int64_t gslot, uint32_t* scratch, const uint32_t* svs,
                                               const int (&start)[2]) {
  using TS = TbShape<C, T>;
  const int L = a.L;
  const int lane = threadIdx.x & 31;
  const int tau = lane & (T - 1);
  const unsigned gmask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
  __syncwarp(gmask);  // the forward pass's shared memory is reused by the ring
  uint32_t* ring = scratch + tau * TS::RING_WORDS;
  if constexpr (T == 1) {
    // both PBs of the pair, exact walks from S_0 at their last stages
    const int jA = gA.iend - L, jB = hasB ? gB.iend - L : -1;
    const int emit_top[2] = {min(jA, gA.nout - 1), min(jB, gB.nout - 1)};
    const int jend[2] = {jA, jB};
    const int x[2] = {0, 1};
    const int nout[2] = {gA.nout, gB.nout};
    uint8_t* const dst[2] = {gA.dst, gB.dst};
    int psi[2] = {start[0], start[1]}, g[2];
    tb_walk_any<C, T, SMEM, 2>(a, gslot, svs, ring, L, max(jA, jB), 0, emit_top, jend, x, nout, dst, -1, psi, g);
  } else {
    // Segments: lane tau walks segment tau of the records of both PBs of
    // the pair (two chains over the same records: two independent dependency
    // chains per lane, one record stream; measured faster than half the
    // lanes per PB at two and four threads per pair).
    const int jA = gA.iend - L, jB = hasB ? gB.iend - L : -1;
    const int s = tau;
    const int jtop = max(jA, jB);
    // Segment length (whole bytes): a lower segment is walked with LAMBDA
    // records of warm-up above it and the top one exactly, so the lower
    // segments take (J - LAMBDA) / T records each and the top one the rest,
    // which evens out the lanes' walks (K=7, D = 512, L = 42: 304 and 306
    // records at two threads per pair instead of 336 and 274).  Below
    // 2 LAMBDA records the even split J / T is kept: at low Eb/N0 a walk
    // from the exact state then often has not met the first walk's path by
    // the end of so short a segment, and every such exit sends the segment
    // below to a serial re-walk (eight threads per pair at 0 dB: 0.414
    // against 0.393 ms).
    const int seg_bal = (((jtop + 1 - TS::LAMBDA) / T) + 4) & ~7;
    const int seg = seg_bal >= 2 * TS::LAMBDA ? seg_bal : (((jtop + 1 + T - 1) / T) + 7) & ~7;
    const int stop = min(T - 1, jtop / seg);  // top non-empty segment
    const int lo = s * seg;
    const int hi = (s == stop) ? jtop : min(jtop, lo + seg - 1);
    const bool active = lo <= jtop;
    const int hs = (s == stop) ? jtop : min(jtop, hi + TS::LAMBDA);
    // a walk that begins at its PB's last record starts exactly; the others
    // begin with a guess (the same state), checked below
    int psi[2] = {start[0], start[1]}, g[2] = {0, 0};
    if (active) {
      const int emit_top[2] = {min(hi, gA.nout - 1), min(hi, gB.nout - 1)};
      const int je[2] = {jA, jB};
      const int x[2] = {0, 1};
      const int nout[2] = {gA.nout, gB.nout};
      uint8_t* const dst[2] = {gA.dst, gB.dst};
      tb_walk_any<C, T, SMEM, 2>(a, gslot, svs, ring, L, hs, lo, emit_top, je, x, nout, dst, hi, psi, g);
    }
    // One parallel round first: every guessed segment whose entry state
    // differs from the exit state of the first walk of the segment above is
    // walked again from that state, all such segments at once in their own
    // lanes, and both PBs of a lane in one two-chain walk over their common
    // records (a chain that needs no second walk writes nothing).  The exit
    // of a segment above is exact unless that segment was itself walked
    // again and ended elsewhere, which the top-down check below finds (and
    // walks again, one segment after another) as before.
    if constexpr (PAR) {
      const int topA = min(T - 1, jA / seg), topB = hasB ? min(T - 1, jB / seg) : -1;
      const int src = (tau + 1) & (T - 1);
      const int aboveA = __shfl_sync(gmask, psi[0], src, T);
      const int aboveB = __shfl_sync(gmask, psi[1], src, T);
      const bool redoA = tau < topA && aboveA != g[0];
      const bool redoB = hasB && tau < topB && aboveB != g[1];
      if (redoA || redoB) {
        const int lo_q = tau * seg;
        const int hiA = min(jA, lo_q + seg - 1), hiB = min(jB, lo_q + seg - 1);
        int p2[2] = {aboveA, aboveB}, g2[2];
        const int emit_top[2] = {redoA ? min(hiA, gA.nout - 1) : -1, redoB ? min(hiB, gB.nout - 1) : -1};
        const int je[2] = {jA, jB};
        const int x[2] = {0, 1};
        const int nout[2] = {gA.nout, gB.nout};
        uint8_t* const dst[2] = {gA.dst, gB.dst};
        const int hs2 = max(redoA ? hiA : -1, redoB ? hiB : -1);
        tb_walk_any<C, T, SMEM, 2>(a, gslot, svs, ring, L, hs2, lo_q, emit_top, je, x, nout, dst, -1, p2, g2);
        if (redoA) {
          psi[0] = p2[0];
          g[0] = aboveA;
        }
        if (redoB) {
          psi[1] = p2[1];
          g[1] = aboveB;
        }
      }
    }
    // top-down check of the guessed segments of each PB: segment q is exact
    // if the state its walk held at record hi_q equals the exact exit state
    // of segment q + 1; otherwise it is walked again from that state (rare).
    // A chain whose last record lies in segment q started there exactly.
    for (int pb = 0; pb < (hasB ? 2 : 1); ++pb) {
      const PbRun& gp = pb ? gB : gA;
      const int jend_p = pb ? jB : jA;
      const int seg_p = seg;
      const int top = min(T - 1, jend_p / seg_p);
      const int base = 0;  // lane of segment 0
      const int c = pb;    // chain of this PB in every lane
      int exact = __shfl_sync(gmask, c ? psi[1] : psi[0], base + top, T);
      for (int q = top - 1; q >= 0; --q) {
        const int gq = __shfl_sync(gmask, c ? g[1] : g[0], base + q, T);
        int ex = __shfl_sync(gmask, c ? psi[1] : psi[0], base + q, T);
        if (gq != exact) {
          if (tau == base + q) {
            // the same prefetched walk as above, from the exact state
            const int lo_q = q * seg_p, hi_q = min(jend_p, lo_q + seg_p - 1);
            int p2[1] = {exact}, g2[1];
            const int emit_top[1] = {min(hi_q, gp.nout - 1)};
            const int je[1] = {jend_p};
            const int x[1] = {pb};
            const int nout[1] = {gp.nout};
            uint8_t* const dst[1] = {gp.dst};
            tb_walk_any<C, T, SMEM, 1>(a, gslot, svs, ring, L, hi_q, lo_q, emit_top, je, x, nout, dst, -1, p2, g2);
            if (c) psi[1] = p2[0]; else psi[0] = p2[0];
          }
          ex = __shfl_sync(gmask, c ? psi[1] : psi[0], base + q, T);
        }
        exact = ex;
      }
    }
  }
}

// VAR: honour the traceback and frame variants of KArgs (argmin start state,
// tail-biting windows); the batch kernel decodes the plain scheme only.
// PAR: see traceback_pair.
template <class C, int T, bool PUNCT, bool SMEM, bool VAR = false, bool PAR = true>
__device__ __forceinline__ void decode_pair(const KArgs& a, const PairWork& wk, int64_t gslot,
                                            uint32_t* __restrict__ scratch, uint32_t* __restrict__ svs) {
  using S = Shape<C, T>;
  constexpr int R = C::R;
  constexpr int M = S::M, P = S::P, CH = S::CH;
  const int lane = threadIdx.x & 31;
  const int tau = lane & (T - 1);
  const unsigned gmask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
  const int L = a.L;

  PbRun gA = pb_run<R, VAR>(a, wk.A.llr, wk.A.out, wk.A.n, wk.A.b);
  PbRun gB = wk.hasB ? pb_run<R, VAR>(a, wk.B.llr, wk.B.out, wk.B.n, wk.B.b) : gA;
  if (!wk.hasB) gB.iend = -1;
  const int I = max(gA.iend, gB.iend) + 1;  // lock-step stages
  const int J = I - L;                      // survivor records (stages L..I-1)

  // soft-value staging: raw chunk c of PB A / B in buffer c & 1
  constexpr int CB = raw_chunk_bytes<C>(CH);
  int8_t* raw = reinterpret_cast<int8_t*>(scratch + raw_offset_words<C, T>());
  const int nchunk = (I + CH - 1) / CH;
  // relative value index at byte 0 of raw buffers 0 / 1 of PB A / B
  int cbA0 = stage_raw_chunk<R, CH>(a, gA, wk.A.llr, wk.A.llr_end, 0, raw, tau, T);
  int cbB0 = stage_raw_chunk<R, CH>(a, gB, wk.B.llr, wk.B.llr_end, 0, raw + CB, tau, T);
  int cbA1 = 0, cbB1 = 0;
  asm volatile("cp.async.commit_group;" ::: "memory");

  uint32_t sel[P][3];
#pragma unroll
  for (int ph = 0; ph < P; ++ph) {
    const uint32_t m = thread_swap<C, T>(tau, ph);
#pragma unroll
    for (int q = 0; q < 3; ++q) sel[ph][q] = 0u - ((m >> (R - 1 - q)) & 1u);
  }

  uint32_t pm[M];
#pragma unroll
  for (int k = 0; k < M; ++k) pm[k] = 0u;
  if (gA.delta == 0) reinit_lane<C, T>(pm, tau, 0x0000ffffu, gA.known_start);
  if (gB.delta == 0 && wk.hasB) reinit_lane<C, T>(pm, tau, 0xffff0000u, gB.known_start);
  // periods [fast_lo, fast_hi] need no per-stage checks
  const int dmax = max(gA.delta, gB.delta);
  const int fast_lo = dmax + (dmax > 0 ? 1 : 0);
  const bool fast_ok = wk.hasB && (PUNCT || R != 2 || (((reinterpret_cast<uintptr_t>(wk.A.llr) |
                                                            reinterpret_cast<uintptr_t>(wk.B.llr)) & 1) == 0));
  // with the argmin start the period holding a PB's last stage is checked,
  // so that its metrics can be captured there
  const int fast_hi = fast_ok ? min(gA.iend, gB.iend) - (P - 1) - ((VAR && a.tb_argmin) ? 1 : 0) : -1;
  int start[2] = {0, 0};

  const int64_t rec_stride = a.surv_pairs * (int64_t)a.surv_rs;  // global: words per record row
  uint32_t* gsv = a.surv + gslot * a.surv_rs + tau * S::W;
  uint32_t* ssv = svs + tau * S::W;

  int since_renorm = 0;
  for (int i0 = 0; i0 < I; i0 += P) {
    if (i0 % CH == 0) {
      // chunk c begins: its raw bytes were requested one chunk ago; request
      // chunk c + 1 into the buffer chunk c - 1 used (every lane is past it)
      const int c = i0 / CH;
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp(gmask);
      if (c + 1 < nchunk) {
        const int nb = (c + 1) & 1;
        const int na = stage_raw_chunk<R, CH>(a, gA, wk.A.llr, wk.A.llr_end, c + 1, raw + nb * 2 * CB, tau, T);
        const int nbb =
            stage_raw_chunk<R, CH>(a, gB, wk.B.llr, wk.B.llr_end, c + 1, raw + nb * 2 * CB + CB, tau, T);
        if (nb) { cbA1 = na; cbB1 = nbb; } else { cbA0 = na; cbB0 = nbb; }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int cur = (i0 / CH) & 1;
    const int8_t* bufA = raw + cur * 2 * CB;
    const int8_t* bufB = bufA + CB;
    const int cbA = cur ? cbA1 : cbA0, cbB = cur ? cbB1 : cbB0;
    const bool fast = i0 >= fast_lo && i0 <= fast_hi;
    if (fast && i0 >= L)
      forward_period<C, T, false, PUNCT, SMEM, true>(pm, sel, a, bufA, cbA, bufB, cbB, wk.hasB, i0, I, L, tau, gA,
                                                     gB, gsv, rec_stride, ssv);
    else if (fast && i0 + P <= L)
      forward_period<C, T, false, PUNCT, SMEM, false>(pm, sel, a, bufA, cbA, bufB, cbB, wk.hasB, i0, I, L, tau, gA,
                                                      gB, gsv, rec_stride, ssv);
    else
      forward_period<C, T, true, PUNCT, SMEM, true, VAR>(pm, sel, a, bufA, cbA, bufB, cbB, wk.hasB, i0, I, L, tau,
                                                         gA, gB, gsv, rec_stride, ssv, start, gmask);
    if (i0 + P < I) {
      // end of a full period: transpose back to psi = u (T > 1)
      if constexpr (vector_transpose<C, T>()) {
        // state u = (tau' << r) | k' comes from thread k' mod T, register
        // (tau' << (r - t)) | (k' >> t)
        constexpr int MT = M / T, STR = M + 4;
        __syncwarp(gmask);
        uint32_t* mine = scratch + tau * STR;
#pragma unroll
        for (int k = 0; k < M; k += 4)
          *reinterpret_cast<uint4*>(mine + k) = make_uint4(pm[k], pm[k + 1], pm[k + 2], pm[k + 3]);
        __syncwarp(gmask);
#pragma unroll
        for (int w = 0; w < T; ++w) {
          const uint32_t* src = scratch + w * STR + tau * MT;
#pragma unroll
          for (int m = 0; m < MT; m += 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(src + m);
            pm[(m + 0) * T + w] = q.x;
            pm[(m + 1) * T + w] = q.y;
            pm[(m + 2) * T + w] = q.z;
            pm[(m + 3) * T + w] = q.w;
          }
        }
      } else if constexpr (T > 1) {
        __syncwarp(gmask);
#pragma unroll
        for (int k = 0; k < M; ++k) scratch[(k << S::t) | tau] = pm[k];
        __syncwarp(gmask);
        const uint32_t* src = scratch + (tau << S::r);
        if constexpr (M >= 4) {
#pragma unroll
          for (int k = 0; k < M; k += 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(src + k);
            pm[k] = q.x; pm[k + 1] = q.y; pm[k + 2] = q.z; pm[k + 3] = q.w;
          }
        } else {
          const uint2 q = *reinterpret_cast<const uint2*>(src);
          pm[0] = q.x; pm[1] = q.y;
        }
      }
      if (++since_renorm == S::RENORM_PERIODS) {
        since_renorm = 0;
        uint32_t ref = pm[0];
        if constexpr (T > 1) ref = __shfl_sync(gmask, ref, 0, T);
#pragma unroll
        for (int k = 0; k < M; ++k) pm[k] = pm[k] + S::RENORM_BASE - ref;
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");

  traceback_pair<C, T, SMEM, PAR>(a, gA, gB, wk.hasB, J, gslot, scratch, svs, start);
}

// Minimum resident CTAs of 256 threads the compiler is asked to allow: 2 (at
// most 128 registers) for the 256-state code at eight threads per pair,
// whose 2049-warp launch for a 2^24-bit stream then fits one wave (16 warps
// per SM) and runs 10% faster without spilling; 1 elsewhere (the other
// instances either use fewer registers anyway or slow down when squeezed).
template <class C, int T>
__host__ __device__ constexpr int decode_min_ctas() {
  return (C::N == 256 && T == 8) ? 2 : 1;
}

// Plain launch: pair p of blocks [b_first, n_blocks) of one stream.  SMEM:
// survivor records of each group in shared memory (a.smem_rec_words words
// per group), else in a.surv.
// VAR: the instance honours the variants of KArgs (argmin traceback start,
// tail-biting windows); the plain instances carry none of that code.  The
// traceback's parallel re-walk round is left out where the launch bounds
// hold the kernel to 128 registers (it spilled there and cost 4.5 % of the
// K=9 stream at eight threads per pair).
template <class C, int T, bool PUNCT, bool SMEM, bool VAR = false>
__global__ void __launch_bounds__(256, decode_min_ctas<C, T>()) pbvd_decode_kernel(const KArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int groups_per_cta = blockDim.x / T;
  const int gl = threadIdx.x / T;
  const int64_t pair = (int64_t)blockIdx.x * groups_per_cta + gl;
  if (pair >= a.n_pairs) return;
  constexpr int SW = scratch_words_per_group<C, T>();
  uint32_t* scratch = smem + gl * SW;
  uint32_t* svs = smem + groups_per_cta * SW + (int64_t)gl * a.smem_rec_words;
  PairWork wk;
  wk.A.llr = a.llr;
  wk.A.llr_end = a.llr + a.llr_count;
  wk.A.out = a.out;
  wk.A.n = a.n;
  wk.A.b = a.b_first + 2 * pair;
  wk.B = wk.A;
  wk.B.b = wk.A.b + 1;
  wk.hasB = wk.B.b < a.n_blocks;
  decode_pair<C, T, PUNCT, SMEM, VAR, decode_min_ctas<C, T>() == 1>(a, wk, pair, scratch, svs);
}

}  // namespace pbvd
