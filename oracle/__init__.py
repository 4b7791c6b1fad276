"""FP64 CPU oracle for the sketched recompression of Tucker sums (arXiv 2603.13532).

TEST INFRASTRUCTURE: a plain, slow, float64 restatement of the paper's method
(Sec. 2-3, Algs. 2-4) used only by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library (``paper_2603_13532_gb300``)
never imports it, and it shares no code with the CUDA path.

Modules
  rng         counter-based Gaussian Omega (Philox4x64-10 + Box-Muller)
  tensor      Kronecker / Khatri-Rao products, unfoldings, TTM, Tucker helpers
  sketch_sum  the method: sketch sizes, structured sketches, QR basis, core
              projection (and its gradient with Q fixed), ST-HOSVD, recompress
  subrank     the effective subrank heuristic (Alg. 5): weighted Gram spectra,
              effective ranks and the sketch sizes they give

Every function is pinned by ``tests/test_oracle_*.py`` against something other
than itself (numpy's Philox, brute-force dense sketches, closed-form recovery,
invariants, finite differences).  Parity unpinned: none of the functions here;
the randomized accuracy of the method itself is not bounded by the paper.
"""
from . import rng, sketch_sum, subrank, tensor  # noqa: F401
