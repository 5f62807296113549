// Kernel instances of the (2,1,7) code with generators (171, 133) octal,
// the code of the paper's experiments (Sec. V), unpunctured.
#include "pbvd_instances.cuh"

namespace pbvd {
using K7 = Code<7, 0171u, 0133u, 0u>;

int register_k7(KernelEntry* out, int cap) {
  const KernelEntry all[] = {make_entry<K7, 1>(), make_entry<K7, 2>(),  make_entry<K7, 4>(),
                             make_entry<K7, 8>(), make_entry<K7, 16>(), make_warp_entry<K7>()};
  int n = 0;
  for (const KernelEntry& e : all)
    if (n < cap) out[n++] = e;
  return n;
}
}  // namespace pbvd
