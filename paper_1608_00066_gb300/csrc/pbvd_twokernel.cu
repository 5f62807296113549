// The paper's own two-kernel design (Sec. IV-A/IV-B, Algorithm 1, Table 1),
// kept as an ablation beside the fused kernel of pbvd_device.cuh.
//
// K1 (forward procedure): a thread block serves 32 PBs with 32 N_c threads.
// The butterflies of the trellis fall into N_c groups by their codeword alpha
// (Sec. III-B, Table 2; the groups are cosets, so all have N/(2 N_c)
// butterflies); warp w serves group w of the block's 32 PBs, thread t of each
// warp PB t.  Per stage a thread computes its group's four branch metrics
// (alpha, beta, gamma, theta of Eqs. (3)-(6)), reads the two predecessor
// metrics of each of its butterflies from shared memory laid out PM[N][32]
// (state major, PB minor: bank-conflict free), computes the two successors
// with their decision bits into one survivor word of N/N_c bits, waits for the
// whole block, stores the new metrics, and writes its survivor word to global
// memory at SP[stage][group][PB] (coalesced over the warp's 32 PBs).
// K2 (backward procedure): one thread per PB walks from S_0 at its last stage
// down to its first decoded stage, loading at every stage the N_c survivor
// words of its PB (each load coalesced over the warp) and picking the bit of
// the current state from the lookup of its group and position.
//
// Metrics are 32-bit integers (no renormalisation); the block geometry, known
// start, tie rule and output packing are those of the fused kernel, so both
// produce the same bits.  Unpunctured codes.
#include <cuda_runtime.h>

#include "pbvd.h"
#include "pbvd_device.cuh"
#include "pbvd_internal.h"

namespace pbvd {
namespace {

// Number of butterfly groups: distinct alpha(2j) over the butterflies.
template <class C>
__host__ __device__ constexpr int group_count() {
  bool seen[8] = {false, false, false, false, false, false, false, false};
  int n = 0;
  for (int j = 0; j < C::N / 2; ++j) {
    const uint32_t a = C::alpha((uint32_t)(2 * j));
    if (!seen[a]) {
      seen[a] = true;
      ++n;
    }
  }
  return n;
}

// Label (alpha) of group g: the g-th smallest alpha that occurs.
template <class C>
__host__ __device__ constexpr uint32_t group_alpha(int g) {
  bool seen[8] = {false, false, false, false, false, false, false, false};
  for (int j = 0; j < C::N / 2; ++j) seen[C::alpha((uint32_t)(2 * j))] = true;
  for (uint32_t a = 0; a < 8; ++a)
    if (seen[a] && g-- == 0) return a;
  return 0;
}

template <class C>
struct TwoShape {
  static constexpr int NC = group_count<C>();       // groups = warps per K1 block
  static constexpr int NB = C::N / 2 / NC;          // butterflies per group
  static constexpr int BITS = 2 * NB;               // survivor bits per thread and stage
  static_assert(BITS <= 32, "one survivor word per group");
  static constexpr uint32_t BIG = 8192u;
};

// Geometry of PB b in lock-step indices (i = L is stage bD), as pb_run.
struct TwoPb {
  int delta, iend, nout, known;
  int64_t v0;  // soft value index of stage f0
};

__device__ __forceinline__ TwoPb two_pb(const KArgs& a, int64_t b, int R) {
  const int64_t n = a.n, D = a.D, L = a.L;
  const int64_t s = b * D - L, e = (b + 1) * D + L;
  const int64_t f0 = s < 0 ? 0 : s;
  const int64_t f1 = (e < n ? e : n) - 1;
  const int64_t o0 = b * D;
  const int64_t o1 = (b + 1) * D < n ? (b + 1) * D : n;
  TwoPb p;
  p.delta = (int)(L - (o0 - f0));
  p.iend = p.delta + (int)(f1 - f0);
  p.nout = (int)(o1 - o0);
  p.known = f0 == 0;
  p.v0 = f0 * R;
  return p;
}

// K1: forward procedure.  sp: SP[i][NC][sp_pbs] words, i = lock-step index.
template <class C>
__global__ void __launch_bounds__(256) two_k1(const KArgs a, uint32_t* __restrict__ sp, int64_t sp_pbs) {
  using S = TwoShape<C>;
  constexpr int N = C::N, R = C::R, HALF = N / 2;
  constexpr uint32_t g0 = C::g0(), gK = C::gK();
  __shared__ int32_t pm_s[N][32];
  const int t = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * 32 + t;
  const bool live = b < a.n_blocks;
  TwoPb g = live ? two_pb(a, b, R) : TwoPb{0, -1, 0, 0, 0};
  // the largest last stage of the block's PBs bounds the lock-step loop
  int iend_blk = g.iend;
  for (int off = 16; off > 0; off >>= 1) iend_blk = max(iend_blk, __shfl_xor_sync(0xffffffffu, iend_blk, off));
  // butterflies of group w, in increasing j (the survivor bit order)
  const uint32_t al = group_alpha<C>(w), be = al ^ gK, ga = al ^ g0, th = al ^ gK ^ g0;
  // (unrolled selects, so that js stays in registers)
  int js[S::NB];
  {
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      const bool m = C::alpha((uint32_t)(2 * j)) == al;
#pragma unroll
      for (int p = 0; p < S::NB; ++p)
        if (m && cnt == p) js[p] = j;
      cnt += m ? 1 : 0;
    }
  }
  const int I = iend_blk + 1;  // the same in every warp: all serve the same 32 PBs
  const int8_t* src = a.llr + g.v0;
  for (int i = 0; i < I; ++i) {
    const bool act = live && i >= g.delta && i <= g.iend;
    int32_t reg[2 * S::NB];
    uint32_t word = 0u;
    if (act) {
      // the four branch metrics of the group (Sec. III-B)
      int32_t d0[3], d1[3];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int l = src[(int64_t)(i - g.delta) * R + r];
        l = l < -127 ? -127 : l;
        d0[r] = 127 - l;  // distance to mu(0) = +127
        d1[r] = 127 + l;  // distance to mu(1) = -127
      }
      auto bm = [&](uint32_t c) {
        int32_t m = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) m += ((c >> (R - 1 - r)) & 1u) ? d1[r] : d0[r];
        return m;
      };
      const int32_t ba = bm(al), bb = bm(be), bg = bm(ga), bt = bm(th);
      const bool init = i == g.delta;
#pragma unroll
      for (int p = 0; p < S::NB; ++p) {
        const int j = js[p];
        int32_t pm1, pm2;
        if (init) {
          pm1 = g.known ? (j == 0 ? 0 : (int32_t)S::BIG) : 0;
          pm2 = g.known ? (int32_t)S::BIG : 0;
        } else {
          pm1 = pm_s[2 * j][t];
          pm2 = pm_s[2 * j + 1][t];
        }
        // Eq. (1): successor j from alpha / gamma, successor j + N/2 from
        // beta / theta; the lower branch is kept only when strictly smaller
        const int32_t u0 = pm1 + ba, l0 = pm2 + bg;
        const int32_t u1 = pm1 + bb, l1 = pm2 + bt;
        reg[2 * p] = l0 < u0 ? l0 : u0;
        reg[2 * p + 1] = l1 < u1 ? l1 : u1;
        word |= (uint32_t)(l0 < u0) << (2 * p);
        word |= (uint32_t)(l1 < u1) << (2 * p + 1);
      }
    }
    __syncthreads();  // every read of this stage's metrics is done
    if (act) {
#pragma unroll
      for (int p = 0; p < S::NB; ++p) {
        pm_s[js[p]][t] = reg[2 * p];
        pm_s[js[p] + HALF][t] = reg[2 * p + 1];
      }
      sp[((int64_t)i * S::NC + w) * sp_pbs + b] = word;
    }
    __syncthreads();  // the new metrics are in place
  }
}

// K2: backward procedure, one thread per PB.
template <class C>
__global__ void __launch_bounds__(256) two_k2(const KArgs a, const uint32_t* __restrict__ sp, int64_t sp_pbs) {
  using S = TwoShape<C>;
  constexpr int N = C::N, HALF = N / 2, v = C::v;
  // lookup tables: group and bit position of each state's decision
  __shared__ uint8_t grp[N], pos[N];
  for (int u = threadIdx.x; u < N; u += blockDim.x) {
    const int j = u & (HALF - 1);
    const uint32_t al = C::alpha((uint32_t)(2 * j));
    int gi = 0;
    while (group_alpha<C>(gi) != al) ++gi;
    int rank = 0;
    for (int jj = 0; jj < j; ++jj)
      if (C::alpha((uint32_t)(2 * jj)) == al) ++rank;
    grp[u] = (uint8_t)gi;
    pos[u] = (uint8_t)(2 * rank + (u >> (v - 1)));
  }
  __syncthreads();
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.n_blocks) return;
  const TwoPb g = two_pb(a, b, C::R);
  const int L = a.L;
  uint8_t* dst = a.out + ((b * a.D) >> 3);
  int state = 0;
  uint32_t acc = 0u;
  for (int i = g.iend; i >= L; --i) {
    uint32_t words[S::NC];
#pragma unroll
    for (int q = 0; q < S::NC; ++q) words[q] = sp[((int64_t)i * S::NC + q) * sp_pbs + b];
    const int k = i - L;  // stage bD + k
    if (k < g.nout) {
      acc = (acc << 1) | (uint32_t)((state >> (v - 1)) & 1);
      if ((k & 7) == 0) dst[k >> 3] = (uint8_t)acc;
    }
    uint32_t word = words[0];
#pragma unroll
    for (int q = 1; q < S::NC; ++q) word = grp[state] == q ? words[q] : word;
    const int bit = (int)((word >> pos[state]) & 1u);
    state = 2 * (state & (HALF - 1)) + bit;
  }
}

template <class C>
cudaError_t launch_two(const KArgs& a, uint32_t* sp, int64_t sp_pbs, cudaStream_t s) {
  using S = TwoShape<C>;
  const int64_t g1 = (a.n_blocks + 31) / 32;
  two_k1<C><<<(unsigned)g1, 32 * S::NC, 0, s>>>(a, sp, sp_pbs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int t2 = 32 * S::NC;
  const int64_t g2 = (a.n_blocks + t2 - 1) / t2;
  two_k2<C><<<(unsigned)g2, t2, 0, s>>>(a, sp, sp_pbs);
  return cudaGetLastError();
}

}  // namespace

// Survivor words per lock-step stage and PB, and the launch, for the codes
// the ablation is built for (K=7 (171,133) and K=9 (557,663,711)); -1 for
// others.
int two_kernel_groups(int K, int R, const uint32_t* gens) {
  if (K == 7 && R == 2 && gens[0] == 0171u && gens[1] == 0133u) return TwoShape<Code<7, 0171u, 0133u, 0u>>::NC;
  if (K == 9 && R == 3 && gens[0] == 0557u && gens[1] == 0663u && gens[2] == 0711u)
    return TwoShape<Code<9, 0557u, 0663u, 0711u>>::NC;
  return -1;
}

cudaError_t two_kernel_launch(int K, const KArgs& a, uint32_t* sp, int64_t sp_pbs, cudaStream_t s) {
  if (K == 7) return launch_two<Code<7, 0171u, 0133u, 0u>>(a, sp, sp_pbs, s);
  return launch_two<Code<9, 0557u, 0663u, 0711u>>(a, sp, sp_pbs, s);
}

}  // namespace pbvd
