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
// Metrics are unsigned 16-bit lanes, renormalised every few stages to
// PM - PM(S_0) + 14336.  The spread of the metrics of one PB never exceeds
// 8192 + v * 254 * R <= 14288 (known start) so after renormalisation they lie
// in [48, 28624] and grow by at most 254 R per stage; with at most 32 stages
// between renormalisations every candidate stays below 65536 and every
// difference of two candidates below 32768, so the 16-bit arithmetic is exact.
//
// Decision bit of output register k: t = Y - X + (0x8000 + BM(gamma) -
// BM(alpha)) per lane, i.e. 0x8000 + (c1 - c0); bit 15 of each lane is set
// iff c1 >= c0 (the upper branch is kept).  Survivor words store that bit
// (1 = upper branch), 16 registers per word: bit k & 15 for PB A and
// 16 + (k & 15) for PB B.  The traceback walks directly in psi coordinates.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pbvd_internal.h"

namespace pbvd {

constexpr uint32_t kSignBias = 0x80008000u;  // 0x8000 in both 16-bit lanes
constexpr uint32_t kRenormBase = 0x38003800u; // 14336 in both lanes
constexpr uint32_t kBigPM = 8192u;            // known-start metric of S_d, d != 0
constexpr uint32_t kLamMax2 = 0x00FE00FEu;    // 254 in both lanes
constexpr int kRenormStages = 32;              // max stages between renormalisations
constexpr int kRing = 16;                      // traceback prefetch: stages per chunk

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

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
  static constexpr int r = C::v - t;        // register-index bits
  static constexpr int M = 1 << r;          // states per thread
  static constexpr int P = (T == 1) ? C::v : r;  // stages per period
  static constexpr int B = M < 16 ? M : 16;  // registers per survivor word
  static constexpr int LB = ilog2(B);
  static constexpr int W = M / B;            // survivor words per thread per stage
  static constexpr int RENORM_PERIODS = (kRenormStages / P) > 0 ? (kRenormStages / P) : 1;
  static_assert(r >= 1, "at least two states per thread");
  static_assert(T <= 32, "a group lives in one warp");
};

// Shared-memory words per group for the transpose / traceback ring, and for
// survivor records in shared-memory mode.
template <class C, int T>
__host__ __device__ constexpr int scratch_words_per_group() {
  using S = Shape<C, T>;
  int tr = (T > 1) ? (C::N + 4) : 0;
  int ring = 2 * kRing * T * S::W;
  int m = tr > ring ? tr : ring;
  return (m + 3) & ~3;
}
template <class C, int T>
__host__ __device__ constexpr int record_words_per_stage() {
  return T * Shape<C, T>::W;
}

// ------------------------------------------------------------- soft input --

// Reads the soft values of one PB stage by stage, inserting erasures (0) at
// punctured positions.  Only stages inside [f0, f1] are read.
struct LlrReader {
  int64_t pos;   // unpunctured: index of the stage's first value
  int col;       // punctured: column s mod P
  int64_t base;  // punctured: index of the first value of the period
};

template <int R>
__device__ __forceinline__ void llr_init(LlrReader& rd, const KArgs& a, int64_t f0) {
  if (a.punct_P == 0) {
    rd.pos = f0 * R;
    rd.col = 0;
    rd.base = 0;
  } else {
    int64_t per = f0 / a.punct_P;
    rd.col = (int)(f0 - per * a.punct_P);
    rd.base = per * a.punct_C;
    rd.pos = 0;
  }
}

// Returns the R values of the current stage (clamped to >= -127 and offset
// by 127, i.e. in [0, 254]) and advances.
template <int R>
__device__ __forceinline__ void llr_next(LlrReader& rd, const KArgs& a, const int8_t* __restrict__ llr,
                                         int (&p)[3]) {
  if (a.punct_P == 0) {
#pragma unroll
    for (int q = 0; q < R; ++q) p[q] = max((int)__ldg(llr + rd.pos + q) + 127, 0);
    rd.pos += R;
  } else {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      int off = a.punct_off[rd.col * 4 + q];
      p[q] = off >= 0 ? max((int)__ldg(llr + rd.base + off) + 127, 0) : 127;
    }
    if (++rd.col == a.punct_P) {
      rd.col = 0;
      rd.base += a.punct_C;
    }
  }
}

// ------------------------------------------------------------ ACS stage --

// Branch metrics of all 2^R codewords for both PBs of the pair, and the
// decision constants kt[c] = 0x8000 + BM(c ^ g0) - BM(c) per lane.  'swp' is
// the thread's codeword relabelling: the butterflies of this thread that sit
// at compile-time register k0 belong to group alpha(k0) ^ swp.
template <class C>
__device__ __forceinline__ void branch_metrics(const uint32_t (&Pk)[3], uint32_t swp,
                                               uint32_t (&bm)[C::NC], uint32_t (&kt)[C::NC]) {
  constexpr int R = C::R;
  uint32_t Pp[3], Mp[3];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    // lane value for code bit 1 is 127 + lambda (distance to -127), for bit 0
    // it is 127 - lambda; relabelling by swp swaps the two.
    uint32_t m1 = Pk[q], m0 = kLamMax2 - Pk[q];
    uint32_t sel = 0u - ((swp >> (R - 1 - q)) & 1u);
    Pp[q] = (m1 & ~sel) | (m0 & sel);
    Mp[q] = (m0 & ~sel) | (m1 & sel);
  }
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

// One trellis stage at phase PH for the thread's M registers (in place).
template <class C, int T, int PH>
__device__ __forceinline__ void acs_stage(uint32_t (&pm)[Shape<C, T>::M], uint32_t (&wd)[Shape<C, T>::W],
                                          const uint32_t (&bm)[C::NC], const uint32_t (&kt)[C::NC]) {
  using S = Shape<C, T>;
  constexpr uint32_t g0 = C::g0(), gK = C::gK();
  uint32_t tt[S::M];
#pragma unroll
  for (int k0 = 0; k0 < S::M; ++k0) {
    if (k0 & (1 << PH)) continue;
    const int k1 = k0 | (1 << PH);
    const uint32_t al = C::alpha(rotr_v<C::v>((uint32_t)k0, PH));
    const uint32_t be = al ^ gK;
    const uint32_t X = pm[k0], Y = pm[k1];
    const uint32_t c0 = X + bm[al], c1 = Y + bm[al ^ g0];
    const uint32_t c2 = X + bm[be], c3 = Y + bm[be ^ g0];
    tt[k0] = Y + kt[al] - X;
    tt[k1] = Y + kt[be] - X;
    pm[k0] = __vminu2(c0, c1);
    pm[k1] = __vminu2(c2, c3);
  }
#pragma unroll
  for (int w = 0; w < S::W; ++w) wd[w] = 0u;
#pragma unroll
  for (int k = 0; k < S::M; ++k) wd[k / S::B] = (wd[k / S::B] >> 1) | (tt[k] & kSignBias);
  if (S::B < 16) {
#pragma unroll
    for (int w = 0; w < S::W; ++w) wd[w] >>= (16 - S::B);
  }
}

// Codeword relabelling of thread tau at phase ph (see branch_metrics).
template <class C, int T>
__device__ __forceinline__ uint32_t thread_swap(int tau, int ph) {
  using S = Shape<C, T>;
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < S::t; ++j)
    if ((tau >> j) & 1) m ^= C::alpha(rotr_v<C::v>(1u << (S::r + j), ph));
  return m;
}

// ------------------------------------------------------------- geometry --

struct PbGeom {
  int64_t f0, f1, o0, o1;
  int delta;  // lock-step index of stage f0
  int iend;   // lock-step index of stage f1
};

__device__ __forceinline__ PbGeom pb_geometry(int64_t n, int D, int L, int64_t b) {
  PbGeom g;
  int64_t s = b * D - L, e = (b + 1) * D + L;
  g.f0 = s < 0 ? 0 : s;
  g.f1 = (e < n ? e : n) - 1;
  g.o0 = b * D;
  g.o1 = (b + 1) * D < n ? (b + 1) * D : n;
  g.delta = (int)(L - (g.o0 - g.f0));
  g.iend = g.delta + (int)(g.f1 - g.f0);
  return g;
}

// ------------------------------------------------------------- the kernel --

template <class C, int T>
__device__ __forceinline__ void reinit_lane(uint32_t (&pm)[Shape<C, T>::M], int tau, uint32_t lane_mask,
                                            bool known_start) {
  using S = Shape<C, T>;
#pragma unroll
  for (int k = 0; k < S::M; ++k) {
    uint32_t init = known_start ? ((tau == 0 && k == 0) ? 0u : (kBigPM | (kBigPM << 16))) : 0u;
    pm[k] = (pm[k] & ~lane_mask) | (init & lane_mask);
  }
}

// Work item of one group: which pair of PBs of which stream.
struct PairWork {
  const int8_t* llr;
  uint8_t* out;
  int64_t n;       // stages of the stream
  int64_t bA;      // first PB of the pair
  bool hasB;       // second PB exists
};

template <class C, int T>
__device__ __forceinline__ void decode_pair(const KArgs& a, const PairWork& wk, int64_t gslot,
                                            uint32_t* __restrict__ scratch, uint32_t* __restrict__ svs) {
  using S = Shape<C, T>;
  constexpr int R = C::R;
  constexpr int M = S::M, W = S::W, P = S::P;
  const int lane = threadIdx.x & 31;
  const int tau = lane & (T - 1);
  const unsigned gmask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
  const int D = a.D, L = a.L;

  const PbGeom gA = pb_geometry(wk.n, D, L, wk.bA);
  const PbGeom gB = wk.hasB ? pb_geometry(wk.n, D, L, wk.bA + 1) : gA;
  const int I = max(gA.iend, gB.iend) + 1;  // lock-step stages
  const int J = I - L;                      // stored survivor records (stages L..I-1)

  LlrReader rA, rB;
  llr_init<R>(rA, a, gA.f0);
  llr_init<R>(rB, a, gB.f0);

  uint32_t swp[P];
#pragma unroll
  for (int ph = 0; ph < P; ++ph) swp[ph] = thread_swap<C, T>(tau, ph);

  uint32_t pm[M];
#pragma unroll
  for (int k = 0; k < M; ++k) pm[k] = 0u;
  if (gA.delta == 0) reinit_lane<C, T>(pm, tau, 0x0000ffffu, gA.f0 == 0);
  if (gB.delta == 0) reinit_lane<C, T>(pm, tau, 0xffff0000u, gB.f0 == 0);

  int64_t rec_stride = a.surv_pairs * (int64_t)(T * W);  // global: words per record row
  uint32_t* gsv = a.surv + gslot * (T * W) + tau * W;
  uint32_t* ssv = svs + tau * W;

  int since_renorm = 0;
  for (int i0 = 0; i0 < I; i0 += P) {
#pragma unroll
    for (int ph = 0; ph < P; ++ph) {
      const int i = i0 + ph;
      if (i < I) {
        if (i == gA.delta && i != 0) reinit_lane<C, T>(pm, tau, 0x0000ffffu, gA.f0 == 0);
        if (i == gB.delta && i != 0 && wk.hasB) reinit_lane<C, T>(pm, tau, 0xffff0000u, gB.f0 == 0);
        int pa[3] = {127, 127, 127}, pb[3] = {127, 127, 127};
        if (i >= gA.delta && i <= gA.iend) llr_next<R>(rA, a, wk.llr, pa);
        if (wk.hasB && i >= gB.delta && i <= gB.iend) llr_next<R>(rB, a, wk.llr, pb);
        uint32_t Pk[3];
#pragma unroll
        for (int q = 0; q < R; ++q) Pk[q] = (uint32_t)pa[q] | ((uint32_t)pb[q] << 16);
        uint32_t bm[C::NC], kt[C::NC];
        branch_metrics<C>(Pk, swp[ph], bm, kt);
        uint32_t wd[W];
        // ph is a compile-time constant after unrolling; dispatch to the
        // matching in-place stage.
        switch (ph) {
          case 0: acs_stage<C, T, 0>(pm, wd, bm, kt); break;
          case 1: if constexpr (P > 1) acs_stage<C, T, (P > 1 ? 1 : 0)>(pm, wd, bm, kt); break;
          case 2: if constexpr (P > 2) acs_stage<C, T, (P > 2 ? 2 : 0)>(pm, wd, bm, kt); break;
          case 3: if constexpr (P > 3) acs_stage<C, T, (P > 3 ? 3 : 0)>(pm, wd, bm, kt); break;
          case 4: if constexpr (P > 4) acs_stage<C, T, (P > 4 ? 4 : 0)>(pm, wd, bm, kt); break;
          case 5: if constexpr (P > 5) acs_stage<C, T, (P > 5 ? 5 : 0)>(pm, wd, bm, kt); break;
          case 6: if constexpr (P > 6) acs_stage<C, T, (P > 6 ? 6 : 0)>(pm, wd, bm, kt); break;
          case 7: if constexpr (P > 7) acs_stage<C, T, (P > 7 ? 7 : 0)>(pm, wd, bm, kt); break;
          default: break;
        }
        if (i >= L) {
          const int j = i - L;
          if (a.smem_surv) {
            uint32_t* d = ssv + j * (T * W);
#pragma unroll
            for (int w = 0; w < W; ++w) d[w] = wd[w];
          } else {
            uint32_t* d = gsv + (int64_t)j * rec_stride;
            if constexpr (W % 4 == 0) {
#pragma unroll
              for (int w = 0; w < W; w += 4)
                *reinterpret_cast<uint4*>(d + w) = make_uint4(wd[w], wd[w + 1], wd[w + 2], wd[w + 3]);
            } else if constexpr (W == 2) {
              *reinterpret_cast<uint2*>(d) = make_uint2(wd[0], wd[1]);
            } else {
              d[0] = wd[0];
            }
          }
        }
      }
    }
    if (i0 + P < I) {
      // end of a full period: transpose back to psi = u (T > 1)
      if constexpr (T > 1) {
        __syncwarp(gmask);
#pragma unroll
        for (int k = 0; k < M; ++k) scratch[(k << S::t) | tau] = pm[k];
        __syncwarp(gmask);
        const uint32_t* src = scratch + (tau << S::r);
        if constexpr (M >= 4) {
#pragma unroll
          for (int k = 0; k < M; k += 4) {
            uint4 q = *reinterpret_cast<const uint4*>(src + k);
            pm[k] = q.x; pm[k + 1] = q.y; pm[k + 2] = q.z; pm[k + 3] = q.w;
          }
        } else {
          uint2 q = *reinterpret_cast<const uint2*>(src);
          pm[0] = q.x; pm[1] = q.y;
        }
      }
      if (++since_renorm == S::RENORM_PERIODS) {
        since_renorm = 0;
        uint32_t ref = pm[0];
        if constexpr (T > 1) ref = __shfl_sync(gmask, ref, 0, T);
#pragma unroll
        for (int k = 0; k < M; ++k) pm[k] = pm[k] + kRenormBase - ref;
      }
    }
  }

  // ---------------------------------------------------------- traceback --
  // Tracer lanes: T == 1: lane walks both PBs; T >= 2: tau 0 -> A, tau 1 -> B.
  constexpr int NCH = (T == 1) ? 2 : 1;
  const bool tracer = (T == 1) || (tau == 0) || (tau == 1 && wk.hasB);
  int psi[NCH], ph[NCH], iend[NCH], nout[NCH];
  int64_t obyte[NCH];
  uint32_t acc[NCH];
  int shift[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int x = (T == 1) ? c : (tau & 1);
    const PbGeom& g = x ? gB : gA;
    psi[c] = 0;
    iend[c] = (x == 1 && !wk.hasB) ? -1 : g.iend;
    ph[c] = (iend[c] >= 0) ? (iend[c] % P) : 0;
    nout[c] = (int)(g.o1 - g.o0);
    obyte[c] = g.o0 >> 3;
    acc[c] = 0u;
    shift[c] = x ? 16 : 0;
  }

  auto walk = [&](int j, const uint32_t* __restrict__ rec) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int i = j + L;
      if (i <= iend[c]) {
        const int p = psi[c];
        const uint32_t w = rec[p >> S::LB];
        const int kept_upper = (w >> (shift[c] + (p & (S::B - 1)))) & 1;
        const int bit = (p >> ph[c]) & 1;
        int np = (p & ~(1 << ph[c])) | ((kept_upper ^ 1) << ph[c]);
        if (ph[c] == 0) {
          np = (int)rotl_v<C::v>((uint32_t)np, P % C::v);
          ph[c] = P - 1;
        } else {
          --ph[c];
        }
        psi[c] = np;
        const int pos = j;  // lock-step index i = L + pos, output stage o0 + pos
        if (pos < nout[c]) {
          acc[c] |= (uint32_t)bit << (pos & 7);
          if ((pos & 7) == 0) {
            wk.out[obyte[c] + (pos >> 3)] = (uint8_t)acc[c];
            acc[c] = 0u;
          }
        }
      }
    }
  };

  if (a.smem_surv) {
    __syncwarp(gmask);
    if (tracer) {
      for (int j = J - 1; j >= 0; --j) walk(j, svs + j * (T * W));
    }
  } else {
    // Double-buffered ring of kRing records per chunk, filled by all T lanes
    // with cp.async, walked by the tracer lanes.
    const int nchunks = (J + kRing - 1) / kRing;
    auto issue = [&](int c, int buf) {
      uint32_t* dst0 = scratch + buf * (kRing * T * W) + tau * W;
      for (int q = 0; q < kRing; ++q) {
        const int j = J - 1 - c * kRing - q;
        if (j < 0) break;
        const uint32_t* src = a.surv + ((int64_t)j * a.surv_pairs + gslot) * (T * W) + tau * W;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(dst0 + q * (T * W));
#pragma unroll
        for (int w = 0; w < W; w += (W >= 4 ? 4 : W)) {
          if constexpr (W >= 4)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 4 * w), "l"(src + w));
          else if constexpr (W == 2)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src));
          else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src));
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    __syncwarp(gmask);
    if (nchunks > 0) issue(0, 0);
    for (int c = 0; c < nchunks; ++c) {
      if (c + 1 < nchunks) {
        issue(c + 1, (c + 1) & 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncwarp(gmask);
      if (tracer) {
        const uint32_t* ring = scratch + (c & 1) * (kRing * T * W);
        const int jhi = J - 1 - c * kRing;
        const int jlo = max(0, jhi - kRing + 1);
        for (int j = jhi; j >= jlo; --j) walk(j, ring + (jhi - j) * (T * W));
      }
      __syncwarp(gmask);
    }
  }
}

// Plain launch: pair p of one stream.
template <class C, int T>
__global__ void __launch_bounds__(256) pbvd_decode_kernel(const KArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int groups_per_cta = blockDim.x / T;
  const int gl = threadIdx.x / T;
  const int64_t pair = (int64_t)blockIdx.x * groups_per_cta + gl;
  if (pair >= a.n_pairs) return;
  constexpr int SW = scratch_words_per_group<C, T>();
  uint32_t* scratch = smem + gl * SW;
  uint32_t* svs = smem + groups_per_cta * SW + (int64_t)gl * a.smem_rec_words;
  PairWork wk;
  wk.llr = a.llr;
  wk.out = a.out;
  wk.n = a.n;
  wk.bA = 2 * pair;
  wk.hasB = (2 * pair + 1) < a.n_blocks;
  decode_pair<C, T>(a, wk, pair, scratch, svs);
}

}  // namespace pbvd
