// Kernel instances of small codes: (2,1,3) with generators (7, 5) and
// (2,1,5) with generators (23, 35) octal.
#include "pbvd_instances.cuh"

namespace pbvd {
using K3 = Code<3, 07u, 05u, 0u>;
using K5 = Code<5, 023u, 035u, 0u>;

int register_small(KernelEntry* out, int cap) {
  const KernelEntry all[] = {make_entry<K3, 1>(), make_entry<K3, 2>(), make_entry<K5, 1>(),
                             make_entry<K5, 2>(), make_entry<K5, 4>(), make_entry<K5, 8>()};
  int n = 0;
  for (const KernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}
}  // namespace pbvd
