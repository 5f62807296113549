// Kernel instances of the (2,1,7) (171, 133) code read through a puncture
// pattern (erasures at the punctured positions).
#include "pbvd_instances.cuh"

namespace pbvd {
using K7 = Code<7, 0171u, 0133u, 0u>;

int register_k7_punctured(KernelEntry* out, int cap) {
  const KernelEntry all[] = {make_entry<K7, 1, true>(), make_entry<K7, 2, true>(),  make_entry<K7, 4, true>(),
                             make_entry<K7, 8, true>(), make_entry<K7, 16, true>(), make_warp_entry<K7, true>()};
  int n = 0;
  for (const KernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}
}  // namespace pbvd
