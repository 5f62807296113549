// Unpacking of q-bit soft values (Sec. IV-C) into the decoder's int8 input.
//
// The paper stores each soft value in q bits, floor(32/q) of them in one
// 32-bit word, to cut the host-to-device transfer (U_1 = 4R / floor(32/q)
// bytes per stage).  Value i sits in word i / m (m = floor(32/q)) at bits
// [q (i mod m), q (i mod m) + q) as a q-bit two's complement number; q = 1
// carries hard decisions (bit 1 = received code bit 1).
//
// The decoder's branch metric on q-bit values is sum_r |lambda_r - mu(c_r)|
// with mu = +-Q, Q = 2^{q-1} - 1 (Q = 1 for hard decisions, twice the Hamming
// distance).  Multiplying every value by s = floor(127 / Q) (after clamping at
// -Q) gives int8 values whose metric with mu = +-127 is s BM_q + (127 - sQ) R
// in every stage: a positive-affine map of all branch metrics of a stage, so
// the add-compare-select takes the same decisions, ties included, and the int8
// kernels decode the q-bit stream bit for bit as the q-bit metric would.
#include <cuda_runtime.h>

#include "pbvd_internal.h"

namespace pbvd {
namespace {

// Each thread writes 16 consecutive output values with one 16-byte store
// (plain stores for the ragged end).  Values [v0, v1) of the packed stream
// go to out[v0 .. v1) (out is indexed by value, as the decoder reads it).
template <int Q_BITS>
__global__ void __launch_bounds__(256) unpack_kernel(const uint32_t* __restrict__ words, int64_t v0, int64_t v1,
                                                     int8_t* __restrict__ out) {
  constexpr int M = 32 / Q_BITS;
  constexpr int QMAX = Q_BITS == 1 ? 1 : (1 << (Q_BITS - 1)) - 1;
  constexpr int S = 127 / QMAX;
  const int64_t base = (v0 & ~(int64_t)15) + 16 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (base >= v1) return;
  uint32_t packed[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    uint32_t acc = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t i = base + 4 * g + b;
      int val = 0;
      if (i >= v0 && i < v1) {
        const uint32_t w = __ldg(words + i / M);
        const uint32_t u = (w >> (Q_BITS * (int)(i % M))) & ((1u << Q_BITS) - 1u);
        if (Q_BITS == 1) {
          val = u ? -S : S;
        } else {
          int x = (int)u - (int)((u >> (Q_BITS - 1)) << Q_BITS);  // sign-extend
          x = x < -QMAX ? -QMAX : x;
          val = x * S;
        }
      }
      acc |= (uint32_t)(uint8_t)(int8_t)val << (8 * b);
    }
    packed[g] = acc;
  }
  if (base >= v0 && base + 16 <= v1 && (reinterpret_cast<uintptr_t>(out + base) & 15) == 0) {
    *reinterpret_cast<uint4*>(out + base) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  } else {
    for (int k = 0; k < 16; ++k) {
      const int64_t i = base + k;
      if (i >= v0 && i < v1) out[i] = (int8_t)(packed[k >> 2] >> (8 * (k & 3)));
    }
  }
}

template <int Q_BITS>
cudaError_t launch_q(const uint32_t* words, int64_t v0, int64_t v1, int8_t* out, cudaStream_t s) {
  const int64_t first = v0 & ~(int64_t)15;
  const int64_t threads = (v1 - first + 15) / 16;
  const int64_t grid = (threads + 255) / 256;
  if (grid <= 0) return cudaSuccess;
  unpack_kernel<Q_BITS><<<(unsigned)grid, 256, 0, s>>>(words, v0, v1, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_unpack(int q, const uint32_t* words, int64_t v0, int64_t v1, int8_t* out, cudaStream_t s) {
  switch (q) {
    case 1: return launch_q<1>(words, v0, v1, out, s);
    case 2: return launch_q<2>(words, v0, v1, out, s);
    case 3: return launch_q<3>(words, v0, v1, out, s);
    case 4: return launch_q<4>(words, v0, v1, out, s);
    case 5: return launch_q<5>(words, v0, v1, out, s);
    case 6: return launch_q<6>(words, v0, v1, out, s);
    case 7: return launch_q<7>(words, v0, v1, out, s);
    case 8: return launch_q<8>(words, v0, v1, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pbvd
