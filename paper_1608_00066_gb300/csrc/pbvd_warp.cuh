// Latency kernel for the 64-state codes: one warp per pair of PBs.
//
// The throughput kernels give each thread many states and move them between
// threads through shared memory once per period; with few PBs in flight (a
// single frame, a short launch) each PB then advances at the speed of one
// long dependency chain.  Here lane j owns butterfly j at every stage: the
// path metrics of states 2j and 2j+1 (natural order, PB A in the low and PB
// B in the high 16 bits) enter, the successors j and j + 32 leave (Sec.
// III-B butterfly, Eq. (1)), and the next stage's inputs are fetched from
// lanes 2j mod 32 and 2j+1 mod 32 with four shuffles.  Lane j keeps the four
// decisions of its butterfly for eight consecutive records in one word (byte
// 2h + x for successor j + 32h of PB x, bit = record mod 8; a set bit means
// the upper branch, the one from S_2j, was kept) and stores it once per
// eight records: block m of a pair's records is 32 words, word j from lane
// j.  The traceback needs no layout arithmetic: the survivor bit of state u
// at record r is bit 8 (2 (u >> 5) + x) + (r & 7) of word u & 31 of block
// r >> 3, the predecessor is 2 (u mod 32) + (1 - bit) and the decoded bit is
// u >> 5 (Algorithm 1).  Sixteen lanes walk each PB in
// speculative byte-aligned segments (each checked against the exact exit
// state of the segment above and re-walked on a mismatch, so the result is
// exact).
#pragma once

#include "pbvd_device.cuh"

namespace pbvd {

constexpr int kWarpCH = 64;       // stages per staged soft-value chunk
constexpr int kWarpU = 8;         // stages per unrolled block
constexpr int kWarpLambda = 56;   // warm-up records of a guessed segment (8K)

// Per-warp shared memory: the raw soft values of two chunks of both PBs, and
// the codeword metrics of the current chunk (NC words per stage).
template <class C>
__host__ __device__ constexpr int warp_raw_words() {
  return (2 * 2 * raw_chunk_bytes<C>(kWarpCH)) / 4;
}
template <class C>
__host__ __device__ constexpr int warp_scratch_words() {
  return warp_raw_words<C>() + kWarpCH * C::NC;
}

// Soft values of both PBs' code bits at lock-step stage i, packed as
// 127 + lambda per 16-bit lane (0 outside a PB's forward range and at
// punctured positions), read from the staged chunk buffers.
template <int R, bool PUNCT>
__device__ __forceinline__ void warp_stage_soft(const KArgs& a, const PbRun& g, const int8_t* buf, int cb, int i,
                                                uint32_t (&u)[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) u[q] = 0u;
  if (g.iend < 0 || i < g.delta || i > g.iend) return;
  const int k = i - g.delta;
  const uint8_t* p = reinterpret_cast<const uint8_t*>(buf) + (rel_value_index<R>(a, g.f0mod, k) - cb);
  if constexpr (!PUNCT) {
#pragma unroll
    for (int q = 0; q < R; ++q) u[q] = p[q];
  } else {
    const int x = g.f0mod + k;
    const int col = x - (x / a.punct_P) * a.punct_P;
    int used = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int off = a.punct_off[col * 4 + q];
      u[q] = off >= 0 ? (uint32_t)p[used] : 0u;
      used += off >= 0;
    }
  }
}

// One stage for both PBs of the pair.  X, Y: metrics of states 2j, 2j+1.
// bm_al: metric of the lane's codeword alpha(2j); bm_co = 254 R - bm_al is
// that of its complement, the codeword of the other three branches' pairs
// (beta = gamma = ~alpha, theta = alpha when every generator taps both ends).
// Returns the lane's four decisions as 0x00 / 0xFF bytes (byte 2h + x: state
// j + 32h of PB x kept its upper branch).
template <class C>
__device__ __forceinline__ uint32_t warp_acs(uint32_t& X, uint32_t& Y, uint32_t bm_al, int lane) {
  constexpr uint32_t SUM = (uint32_t)(254 * C::R) * 0x00010001u;
  const uint32_t bm_co = SUM - bm_al;
  const uint32_t c1 = Y + bm_co, c3 = Y + bm_al;
  const uint32_t n0 = __viaddmin_s16x2(X, bm_al, c1);   // state j
  const uint32_t n1 = __viaddmin_s16x2(X, bm_co, c3);   // state j + 32
  // inputs of the next stage first (the dependency chain): states 2j and
  // 2j+1 live in lanes 2j mod 32 and 2j+1 mod 32, as their successor j
  // (lanes j < 16) or j + 32 (j >= 16)
  const int s0 = (2 * lane) & 31, s1 = (2 * lane + 1) & 31;
  const uint32_t a0 = __shfl_sync(0xffffffffu, n0, s0), a1 = __shfl_sync(0xffffffffu, n1, s0);
  const uint32_t b0 = __shfl_sync(0xffffffffu, n0, s1), b1 = __shfl_sync(0xffffffffu, n1, s1);
  // t = 0x8000 + (lower candidate - upper candidate) per lane
  const uint32_t t0 = c1 + kSignBias - X - bm_al;
  const uint32_t t1 = c3 + kSignBias - X - bm_co;
  X = lane < 16 ? a0 : a1;
  Y = lane < 16 ? b0 : b1;
  return decision_bytes(t0, t1);
}

// Known-start or zero metrics for one PB's half of the lane's two states.
__device__ __forceinline__ void warp_reinit(uint32_t& X, uint32_t& Y, int lane, uint32_t mask, bool known) {
  const uint32_t big = kBigPM | (kBigPM << 16);
  const uint32_t x0 = known ? (lane == 0 ? 0u : big) : 0u;
  const uint32_t y0 = known ? big : 0u;
  X = (X & ~mask) | (x0 & mask);
  Y = (Y & ~mask) | (y0 & mask);
}

template <class C, bool PUNCT, bool SMEM>
__device__ __forceinline__ void warp_decode_pair(const KArgs& a, const PairWork& wk, int64_t gslot,
                                                 uint32_t* __restrict__ scratch, uint32_t* __restrict__ svs) {
  static_assert(C::v == 6, "one butterfly per lane: 64 states");
  static_assert(C::g0() == (uint32_t)C::NC - 1u && C::gK() == (uint32_t)C::NC - 1u,
                "every generator taps the input and the oldest cell");
  constexpr int R = C::R, CH = kWarpCH, U = kWarpU;
  constexpr int CB = raw_chunk_bytes<C>(CH);
  const int lane = threadIdx.x & 31;
  const int L = a.L;

  PbRun gA = pb_run<R>(a, wk.A.llr, wk.A.out, wk.A.n, wk.A.b);
  PbRun gB = wk.hasB ? pb_run<R>(a, wk.B.llr, wk.B.out, wk.B.n, wk.B.b) : gA;
  if (!wk.hasB) gB.iend = -1;
  const int I = max(gA.iend, gB.iend) + 1;

  // the lane's codeword: alpha = c(S_2j, 0), code bit 1 most significant
  const uint32_t al = C::alpha((uint32_t)(2 * lane));

  int8_t* raw = reinterpret_cast<int8_t*>(scratch);
  const int nchunk = (I + CH - 1) / CH;
  int cbA0 = stage_raw_chunk<R, CH>(a, gA, wk.A.llr, wk.A.llr_end, 0, raw, lane, 32);
  int cbB0 = stage_raw_chunk<R, CH>(a, gB, wk.B.llr, wk.B.llr_end, 0, raw + CB, lane, 32);
  int cbA1 = 0, cbB1 = 0;
  asm volatile("cp.async.commit_group;" ::: "memory");

  uint32_t X = 0u, Y = 0u;
  if (gA.delta == 0) warp_reinit(X, Y, lane, 0x0000ffffu, gA.known_start);
  if (gB.delta == 0 && wk.hasB) warp_reinit(X, Y, lane, 0xffff0000u, gB.known_start);
  // block m of the pair's records: svs + 32 m (shared) or gsv + 32 m
  // surv_pairs (global, pair slots interleaved block by block)
  const int64_t blk_stride = 32 * a.surv_pairs;
  uint32_t* gsv = a.surv + gslot * 32;
  uint32_t dacc = 0u;
  const int cs = (8 - (L & 7)) & 7;   // (i0 - L) & 7 for i0 a multiple of 8
  const int us = (L + 7) & 7;         // u with (i0 + u - L) & 7 == 7
  constexpr int RENORM_BLOCKS = Shape<C, 1>::RENORM_STAGES / U;
  static_assert(RENORM_BLOCKS >= 1, "renormalisation interval shorter than a block");
  constexpr uint32_t RENORM_BASE = Shape<C, 1>::RENORM_BASE;
  int since_renorm = 0;

  uint32_t* tab = scratch + warp_raw_words<C>();   // [stage of chunk][codeword]
  for (int i0 = 0; i0 < I; i0 += U) {
    if (i0 % CH == 0) {
      const int c = i0 / CH;
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();
      // codeword metrics of the chunk's stages, two stages per lane
      {
        const int cur = c & 1;
        const int8_t* bufA = raw + cur * 2 * CB;
        const int8_t* bufB = bufA + CB;
        const int cbA = cur ? cbA1 : cbA0, cbB = cur ? cbB1 : cbB0;
#pragma unroll
        for (int h = 0; h < CH / 32; ++h) {
          const int sl = lane + 32 * h;
          const int i = i0 + sl;
          uint32_t ua[3], ub[3], pk[3];
          warp_stage_soft<R, PUNCT>(a, gA, bufA, cbA, i, ua);
          warp_stage_soft<R, PUNCT>(a, gB, bufB, cbB, i, ub);
#pragma unroll
          for (int q = 0; q < 3; ++q) pk[q] = q < R ? pack_soft(ua[q], ub[q]) : 0u;
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
        const int nb = (c + 1) & 1;
        const int na = stage_raw_chunk<R, CH>(a, gA, wk.A.llr, wk.A.llr_end, c + 1, raw + nb * 2 * CB, lane, 32);
        const int nbb = stage_raw_chunk<R, CH>(a, gB, wk.B.llr, wk.B.llr_end, c + 1, raw + nb * 2 * CB + CB, lane, 32);
        if (nb) { cbA1 = na; cbB1 = nbb; } else { cbA0 = na; cbB0 = nbb; }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // metric of the lane's codeword alpha at each stage of the block
    uint32_t bmv[U];
    const uint32_t* trow = tab + (i0 % CH) * C::NC + al;
#pragma unroll
    for (int u = 0; u < U; ++u) bmv[u] = trow[u * C::NC];
    // blocks wholly inside [L, I - 1) that hold no PB's first stage run without
    // per-stage checks: record r = i - L has r & 7 = (cs + u) & 7, and the
    // word of a block of eight records is complete at u == us
    // (the last block always runs checked: it stores the final, partial word)
    const bool plain = i0 >= L && i0 + U < I && (gA.delta < i0 || gA.delta >= i0 + U) &&
                       (!wk.hasB || gB.delta < i0 || gB.delta >= i0 + U);
    if (plain) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t d = warp_acs<C>(X, Y, bmv[u], lane);
        const uint32_t col = 0x01010101u << ((cs + u) & 7);
        dacc = (dacc & ~col) | (d & col);
        if (u == us) {
          const int m = (i0 + u - L) >> 3;
          if constexpr (SMEM) svs[(int64_t)m * 32 + lane] = dacc;
          else gsv[(int64_t)m * blk_stride + lane] = dacc;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u;
        if (i >= I) break;
        if (i == gA.delta && i != 0) warp_reinit(X, Y, lane, 0x0000ffffu, gA.known_start);
        if (i == gB.delta && i != 0) warp_reinit(X, Y, lane, 0xffff0000u, gB.known_start);
        const uint32_t d = warp_acs<C>(X, Y, bmv[u], lane);
        if (i >= L) {
          const int r = i - L;
          const uint32_t col = 0x01010101u << (r & 7);
          dacc = (dacc & ~col) | (d & col);
          if ((r & 7) == 7 || i == I - 1) {
            if constexpr (SMEM) svs[(int64_t)(r >> 3) * 32 + lane] = dacc;
            else gsv[(int64_t)(r >> 3) * blk_stride + lane] = dacc;
          }
        }
      }
    }
    // renormalise every RENORM_BLOCKS blocks (at most RENORM stages apart)
    if (++since_renorm == RENORM_BLOCKS) {
      since_renorm = 0;
      const uint32_t ref = __shfl_sync(0xffffffffu, X, 0);  // state 0
      X = X + RENORM_BASE - ref;
      Y = Y + RENORM_BASE - ref;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();

  // traceback: lanes 0-15 walk PB A, lanes 16-31 PB B, in 16 segments each
  const int xb = lane >> 4, q = lane & 15;
  const PbRun& gp = xb ? gB : gA;
  const int jtop = gp.iend - L;   // top record (-1: no such PB)
  const int seg = (((jtop + 1 + 15) / 16) + 7) & ~7;
  const int lo = q * seg;
  const int hi = min(jtop, lo + seg - 1);
  const int top = seg > 0 ? jtop / seg : 0;
  const bool active = jtop >= 0 && lo <= jtop;
  const int hs = (q == top) ? jtop : min(jtop, hi + kWarpLambda);
  const int emit_top = min(hi, gp.nout - 1);
  auto walk = [&](int from, int to, uint32_t u, int g_at, uint32_t& g) -> uint32_t {
    uint32_t acc = 0u;
    for (int j = from; j >= to; --j) {
      const uint32_t* blk = SMEM ? svs + (int64_t)(j >> 3) * 32 : gsv + (int64_t)(j >> 3) * blk_stride;
      const uint32_t word = blk[u & 31u];
      if (j == g_at) g = u;
      const uint32_t upper = (word >> (((u >> 5) * 2 + xb) * 8 + (j & 7))) & 1u;
      acc = (acc << 1) | (u >> 5);
      u = ((u << 1) & 62u) | (upper ^ 1u);
      if ((j & 7) == 0 && j <= emit_top) {
        const int rem = gp.nout - j;
        const uint32_t keep = rem >= 8 ? 0xffu : ((1u << (rem > 0 ? rem : 0)) - 1u);
        gp.dst[j >> 3] = (uint8_t)(acc & keep);
      }
    }
    return u;
  };
  uint32_t ex = 0u, g = 0u;
  if (active) ex = walk(hs, lo, 0u, hi, g);
  // top-down check of each PB's guessed segments (lanes of the same half)
  const int base = xb * 16;
  const int top_b = __shfl_sync(0xffffffffu, top, base);
  const bool act_b = __shfl_sync(0xffffffffu, active ? 1 : 0, base) != 0;
  uint32_t exact = __shfl_sync(0xffffffffu, ex, base + top_b);
  for (int k = 14; k >= 0; --k) {
    // every lane runs the loop; lanes of the half whose PB has segment k
    // below its top take part
    const uint32_t gk = __shfl_sync(0xffffffffu, g, base + k);
    uint32_t exk = __shfl_sync(0xffffffffu, ex, base + k);
    const bool live = act_b && k < top_b;
    const bool redo = live && gk != exact;
    if (redo && q == k) {
      uint32_t dummy = 0u;
      ex = walk(hi, lo, exact, -1, dummy);
    }
    exk = __shfl_sync(0xffffffffu, ex, base + k);
    if (live) exact = exk;
  }
}

// Plain launch of the warp kernel: pair p of blocks [b_first, n_blocks).
template <class C, bool PUNCT, bool SMEM>
__global__ void __launch_bounds__(256, 1) pbvd_warp_kernel(const KArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int groups_per_cta = blockDim.x / 32;
  const int gl = threadIdx.x / 32;
  const int64_t pair = (int64_t)blockIdx.x * groups_per_cta + gl;
  if (pair >= a.n_pairs) return;
  constexpr int SW = warp_scratch_words<C>();
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
  warp_decode_pair<C, PUNCT, SMEM>(a, wk, pair, scratch, svs);
}

}  // namespace pbvd
