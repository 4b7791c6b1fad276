// Reads "hi lo scale" triples (decimal) from stdin and prints, per line, the bit patterns of
// oz_compose and oz_compose_b (hexadecimal), for tests/test_compose.py.
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "compose.cuh"

int main() {
  long long hi, lo;
  int scale;
  while (std::scanf("%lld %lld %d", &hi, &lo, &scale) == 3) {
    const double a = tks::oz_compose(hi, lo, scale), b = tks::oz_compose_b(hi, lo, scale);
    uint64_t ua, ub;
    std::memcpy(&ua, &a, 8);
    std::memcpy(&ub, &b, 8);
    std::printf("%016" PRIx64 " %016" PRIx64 "\n", ua, ub);
  }
  return 0;
}
