// Prints the tensor-core GEMM's launch shape (csrc/tc_shape.h) over a grid of launches, one line
// each: kmax tiles na nb max_stages allow_two two stages smem acc need, where need is the ring's own
// bytes.
#include <stdio.h>

#include "tc_shape.h"

int main() {
  const int kmaxs[] = {16, 40, 64, 255, 256, 257, 384, 512, 640, 896, 1023, 1024, 1025, 2048, 4000};
  const int tiles[] = {1, 152, 304, 760, 4864, 4865, 15200, 108000};
  for (int km : kmaxs)
    for (int t : tiles)
      for (int na = 1; na <= 3; ++na)
        for (int nb = 1; nb <= 3; ++nb)
          for (int ms = 0; ms <= 4; ++ms)
            for (int al = 0; al <= 1; ++al) {
              const tks::TcShape sh = tks::tc_gemm_shape(km, t, na, nb, ms, al != 0);
              printf("%d %d %d %d %d %d %d %d %zu %d %zu\n", km, t, na, nb, ms, al, sh.two ? 1 : 0, sh.stages,
                     sh.smem, sh.acc, tks::tc_gemm_smem_bytes(sh.stages, na, nb, tks::kTcBN));
            }
  return 0;
}
