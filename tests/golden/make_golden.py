"""Writes the stored expected values under tests/golden/ by calling only oracle/.

  omega_head.json   first draws of Omega_j (hex floats) for a few (seed, problem, mode):
                    float64 draws, float32 draws and their bfloat16 roundings (low-precision
                    sketch); definition: oracle/rng.py (Philox4x64-10 + Box-Muller, Sec. 3.1)
  sketch_sizes.json sketch sizes from Eq. heuristic_formula (Kronecker, integer form) and
                    s = max ell (Khatri-Rao, Sec. 3.2) for the measured workloads

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import rng, sketch_sum  # noqa: E402


def main():
    heads = []
    for seed, problem, mode in [(20260315, 0, 0), (20260315, 0, 2), (20260315, 5, 1), (1, 0, 0)]:
        z = rng.gaussian(seed, problem, mode, np.arange(32))
        z32 = rng.gaussian_f32(seed, problem, mode, np.arange(32))
        zb = rng.round_bf16(z32)
        heads.append(dict(seed=seed, problem=problem, mode=mode,
                          values=[float(x).hex() for x in z],
                          f32_values=[float(x).hex() for x in z32],
                          bf16_values=[float(x).hex() for x in zb]))
    with open(os.path.join(HERE, "omega_head.json"), "w") as f:
        json.dump(dict(source="oracle/rng.py (Philox4x64-10 + Box-Muller)", draws=heads), f, indent=1)

    cases = [("exact_recovery", "kron", [32] * 3), ("decay512", "krp", [58] * 3),
             ("order4-krp", "krp", [48] * 4), ("order4-kron", "kron", [48] * 4),
             ("grad384", "krp", [40] * 3), ("ell-4-4-4", "kron", [4, 4, 4]),
             ("ell-mixed", "kron", [3, 5, 7, 2])]
    out = []
    for name, kind, ell in cases:
        cols, S = sketch_sum.sketch_sizes(kind, ell)
        out.append(dict(name=name, kind=kind, ell=ell, cols=cols, S=S))
    with open(os.path.join(HERE, "sketch_sizes.json"), "w") as f:
        json.dump(dict(source="Eq. heuristic_formula (integer form), Eq. sketch_condition, Sec. 3.2",
                       cases=out), f, indent=1)


if __name__ == "__main__":
    main()
