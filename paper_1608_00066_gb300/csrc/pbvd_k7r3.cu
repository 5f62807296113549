// Kernel instances of the (3,1,7) code with generators (171, 165, 133)
// octal, the rate-1/3 64-state code among the widely used codes of Sec. III-B.
#include "pbvd_instances.cuh"

namespace pbvd {
using K7R3 = Code<7, 0171u, 0165u, 0133u>;

int register_k7_r3(KernelEntry* out, int cap) {
  const KernelEntry all[] = {make_entry<K7R3, 1>(), make_entry<K7R3, 2>(),  make_entry<K7R3, 4>(),
                             make_entry<K7R3, 8>(), make_entry<K7R3, 16>(), make_warp_entry<K7R3>()};
  int n = 0;
  for (const KernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}
}  // namespace pbvd
