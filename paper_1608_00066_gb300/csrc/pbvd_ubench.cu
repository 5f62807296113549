// Integer issue-rate micro-benchmark: how many thread-level operations per
// clock an SM of this device completes for the instructions the decode
// kernels are built from (the 16x2 DPX add-min, three-input add, logic op,
// byte permute, integer multiply-add), alone and mixed across the ALU and FMA
// pipes.  Each thread keeps eight chains that feed each other in a ring
// (new[k] = op(a[k], a[k+1], c)), so no chain can be folded by the compiler
// and every round is eight independent operations that hide latency; 2,048
// threads per SM.  Every CTA records its SM and its start and end clock64;
// an SM's rate is its CTAs' operations over the span from its first start to
// its last end (clock64 counts that SM's cycles, so the result is per clock
// whatever clock the device runs at).
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "pbvd.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kCta = 256;
constexpr int kCtasPerSm = 8;

__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

__device__ __forceinline__ uint32_t add3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("{ .reg .u32 t; add.u32 t, %1, %2; add.u32 %0, t, %3; }" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

__device__ __forceinline__ uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

__device__ __forceinline__ uint32_t perm(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// op 0: 16x2 add-min; 1: three-input add; 2: logic op; 3: byte permute;
// 4: multiply-add; 5: half logic op, half multiply-add; 6: half add-min,
// half multiply-add.
template <int OP>
__device__ __forceinline__ uint32_t ub_op(int k, uint32_t a, uint32_t b, uint32_t c) {
  if constexpr (OP == 0) return __viaddmin_s16x2(a, b, c);
  else if constexpr (OP == 1) return add3(a, b, c);
  else if constexpr (OP == 2) return lop3(a, b, c);
  else if constexpr (OP == 3) return perm(a, b, c);
  else if constexpr (OP == 4) return mad(a, b, c);
  else if constexpr (OP == 5) return (k & 1) ? mad(a, b, c) : lop3(a, b, c);
  else return (k & 1) ? mad(a, b, c) : __viaddmin_s16x2(a, b, c);
}

template <int OP>
__global__ void __launch_bounds__(kCta) ubench_kernel(uint32_t c, int iters, uint32_t* sink, long long* rec) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 0x9E3779B9u + 0x01000193u * (uint32_t)k;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint32_t n[kChains];
#pragma unroll
      for (int k = 0; k < kChains; ++k) n[k] = ub_op<OP>(k, a[k], a[(k + 1) % kChains], c);
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = n[k];
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= a[k];
  if (s == 0x5bd1e995u) sink[0] = s;  // keeps the chains live
  if (threadIdx.x == 0) {
    uint32_t sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    rec[3 * blockIdx.x] = sm;
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = t1;
  }
}

template <int OP>
cudaError_t ub_launch(int grid, int iters, uint32_t* sink, long long* rec) {
  ubench_kernel<OP><<<grid, kCta>>>(0x7fff7fffu, iters, sink, rec);
  return cudaGetLastError();
}

cudaError_t ub_run(int op, int grid, int iters, uint32_t* sink, long long* cycles) {
  switch (op) {
    case 0: return ub_launch<0>(grid, iters, sink, cycles);
    case 1: return ub_launch<1>(grid, iters, sink, cycles);
    case 2: return ub_launch<2>(grid, iters, sink, cycles);
    case 3: return ub_launch<3>(grid, iters, sink, cycles);
    case 4: return ub_launch<4>(grid, iters, sink, cycles);
    case 5: return ub_launch<5>(grid, iters, sink, cycles);
    default: return ub_launch<6>(grid, iters, sink, cycles);
  }
}

}  // namespace

extern "C" PBVD_API int pbvd_measure_int_rate(int op, double* ops_per_clk_per_sm) {
  if (op < 0 || op > 6 || !ops_per_clk_per_sm) return PBVD_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PBVD_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PBVD_ECUDA;
  const int grid = sms * kCtasPerSm;
  uint32_t* sink = nullptr;
  long long* rec = nullptr;
  if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) return PBVD_ENOMEM;
  if (cudaMalloc(&rec, sizeof(long long) * 3 * grid) != cudaSuccess) {
    cudaFree(sink);
    return PBVD_ENOMEM;
  }
  const int iters = 1024;
  cudaError_t e = ub_run(op, grid, 16, sink, rec);  // warm-up
  if (e == cudaSuccess) e = ub_run(op, grid, iters, sink, rec);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<long long> host((size_t)3 * grid);
  if (e == cudaSuccess) e = cudaMemcpy(host.data(), rec, sizeof(long long) * 3 * grid, cudaMemcpyDeviceToHost);
  cudaFree(sink);
  cudaFree(rec);
  if (e != cudaSuccess) return PBVD_ECUDA;
  // per SM: its CTAs' operations over the span of its cycles (SM ids may
  // run past the count of enabled SMs, so index by id)
  const int ids = 4096;
  std::vector<long long> first(ids, -1), last(ids, -1), ctas(ids, 0);
  for (int b = 0; b < grid; ++b) {
    const long long sm = host[3 * b], t0 = host[3 * b + 1], t1 = host[3 * b + 2];
    if (sm < 0 || sm >= ids) continue;
    if (first[sm] < 0 || t0 < first[sm]) first[sm] = t0;
    if (t1 > last[sm]) last[sm] = t1;
    ++ctas[sm];
  }
  const double per_cta = (double)kCta * iters * kUnroll * kChains;
  double sum = 0;
  int used = 0;
  for (int m = 0; m < ids; ++m) {
    if (ctas[m] == 0 || last[m] <= first[m]) continue;
    sum += ctas[m] * per_cta / (double)(last[m] - first[m]);
    ++used;
  }
  if (used == 0) return PBVD_ECUDA;
  *ops_per_clk_per_sm = sum / used;
  return PBVD_OK;
}
