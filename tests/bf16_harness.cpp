// Host build of the bf16 helpers (csrc/bf16.cuh) through tests/host_shim: reads lines "d <hex64>"
// (a float64 to split) or "f <hex32>" (a float32 to split and widen) and prints the three bf16
// planes as hex, then for "f" lines the float64 bits of f32_to_f64_exact.
#include <stdio.h>
#include <string.h>

#include "bf16.cuh"

int main() {
  char kind[4];
  unsigned long long bits;
  while (scanf("%3s %llx", kind, &bits) == 2) {
    uint16_t h0, h1, h2;
    if (kind[0] == 'd') {
      tks::split3(__longlong_as_double((long long)bits), h0, h1, h2);
      printf("%04x %04x %04x\n", h0, h1, h2);
    } else {
      const float v = __uint_as_float((uint32_t)bits);
      tks::split3(v, h0, h1, h2);
      printf("%04x %04x %04x %016llx\n", h0, h1, h2,
             (unsigned long long)__double_as_longlong(tks::f32_to_f64_exact(v)));
    }
  }
  return 0;
}
