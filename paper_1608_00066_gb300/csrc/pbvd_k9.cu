// Kernel instances of the (3,1,9) code with generators (557, 663, 711) octal.
#include "pbvd_instances.cuh"

namespace pbvd {
using K9 = Code<9, 0557u, 0663u, 0711u>;

int register_k9(KernelEntry* out, int cap) {
  const KernelEntry all[] = {make_entry<K9, 4>(), make_entry<K9, 8>(),
                             make_entry<K9, 16>(), make_entry<K9, 32>()};
  int n = 0;
  for (const KernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}
}  // namespace pbvd
