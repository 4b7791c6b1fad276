// Host build of the device RNG (csrc/rng.cuh) through tests/host_shim: reads lines
// "seed problem mode stream block" and prints, per line, the four float64 normals of that Philox
// block and the four float32 normals with their bfloat16 roundings, all as bit patterns (hex).
#include <inttypes.h>
#include <stdio.h>

#include "rng.cuh"

int main() {
  unsigned long long seed, problem, mode, stream, block;
  while (scanf("%llu %llu %llu %llu %llu", &seed, &problem, &mode, &stream, &block) == 5) {
    double z[4];
    float f[4];
    tks::rng::gaussian4(seed, problem, mode, stream, block, z);
    tks::rng::gaussian4_f32(seed, problem, mode, stream, block, f);
    for (int i = 0; i < 4; ++i) printf("%016llx ", (unsigned long long)__double_as_longlong(z[i]));
    for (int i = 0; i < 4; ++i) printf("%08x ", (unsigned)__float_as_uint(f[i]));
    for (int i = 0; i < 4; ++i) printf("%04x%s", (unsigned)tks::rng::f32_to_bf16_bits(f[i]), i < 3 ? " " : "\n");
  }
  return 0;
}
