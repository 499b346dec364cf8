// Independent Philox4x32-10 reference for the oracle's generator: PyTorch's
// at::philox_engine (ATen/core/PhiloxRNGEngine.h), driven so that its internal
// counter equals (ctr0, ctr1, ctr2, ctr3) and its key equals (key0, key1).
// Reads lines "c0 c1 c2 c3 k0 k1" (hex) on stdin, prints the four outputs.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>

int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%x %x %x %x %x %x", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    uint64_t subseq = (uint64_t)c2 | ((uint64_t)c3 << 32);
    uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
    at::philox_engine eng(seed, subseq, offset);
    unsigned r0 = eng(), r1 = eng(), r2 = eng(), r3 = eng();
    std::printf("%08x %08x %08x %08x\n", r0, r1, r2, r3);
  }
  return 0;
}
