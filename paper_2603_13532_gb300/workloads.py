"""Seeded synthetic Tucker-sum workloads (inputs only; none of the method's arithmetic).

Both the CUDA path and the FP64 oracle consume these.  Each builder returns a
``Workload``: a list of independent ``Problem``s (sums of K Tucker terms) and
the method parameters.  Values are float64 arrays; for the mixed-precision
workloads the factors and cores are rounded to bfloat16 values (the tensors
the library receives), so the oracle sees exactly the same numbers.

Synthetic recipes (shapes and distributions of the paper's experiments,
Sec. 5.1, with the sizes of the five workloads the library is measured on):

  exact_recovery   d=3, n=64, K=4, ranks (8,8,8), Haar factors, N(0,1) cores,
                   Kronecker sketch, target 32, oversampling 0, float64
  decay512         d=3, n=512, K=32, ranks ~ U{8..32} per mode; per mode a
                   Haar basis P_m (512 x 128), term factors are random column
                   subsets P_m[:, J_km], core entries z 10^(-(J_k1[a]+J_k2[b]+
                   J_k3[c])/8) so the sum's mode spectra decay like 10^(-i/8);
                   Khatri-Rao sketch, target 48, oversampling 10, bf16 inputs
  order4           d=4, n=256, K=64, ranks ~ U{4..24}, Haar factors, cores
                   N(0,1) 2^(-k/4); target 40, oversampling 8, Kronecker or
                   Khatri-Rao, bf16 inputs
  batched          P=256 independent d=3 sums, n ~ U{128,256,512,1024},
                   K ~ U{8..48}, ranks ~ U{4..32}; target = round-half-up(1.5 x
                   median term rank), oversampling 5, Khatri-Rao, bf16 inputs
  grad384          d=3, n=384, K=16, ranks 16, bf16 factors and cores,
                   Khatri-Rao, target 32 + oversampling 8
  shared_subspace  Sec. 5.1.1 at reduced size: rank-1 terms U_k = Q m_k in a
                   shared rank-10 subspace, oversampling 2
  cancellation     Sec. 5.1.2: target diag(1, .8, .6, 2e-6, 1e-6) plus 30
                   rank-12 noise terms (core diagonals 1e6 .. 1e-5) added with
                   + and - signs
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Problem:
    dims: List[int]
    cores: List[np.ndarray]              # G_k, shape (r_k1, ..., r_kd)
    factors: List[List[np.ndarray]]      # factors[k][m] = U_k^(m), n_m x r_km
    target: List[int]
    oversampling: List[int]
    alpha: Optional[List[float]] = None

    @property
    def order(self):
        return len(self.dims)

    @property
    def num_terms(self):
        return len(self.cores)

    def ranks(self):
        return [list(G.shape) for G in self.cores]

    def terms(self):
        return [(G, Us) for G, Us in zip(self.cores, self.factors)]


@dataclass
class Workload:
    name: str
    problems: List[Problem]
    kind: str                    # "krp" or "kron"
    precision: str               # "fp64" or "mixed"
    seed: int
    tol: float = 0.0
    notes: dict = field(default_factory=dict)


def to_bf16_values(x):
    """Round float64 values to float32 then bfloat16 (both round-to-nearest-even)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    out = (b.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(x))


def haar(rng, n, r):
    """n x r matrix with Haar-distributed orthonormal columns."""
    Q, R = np.linalg.qr(rng.standard_normal((n, r)))
    return Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]


def _finish(problems, bf16):
    if bf16:
        for p in problems:
            p.cores = [to_bf16_values(G) for G in p.cores]
            p.factors = [[to_bf16_values(U) for U in Us] for Us in p.factors]
    return problems


def exact_recovery(seed=20260314, n=64, K=4, r=8, d=3, target=32):
    rng = np.random.default_rng(seed)
    cores = [rng.standard_normal((r,) * d) for _ in range(K)]
    factors = [[haar(rng, n, r) for _ in range(d)] for _ in range(K)]
    p = Problem([n] * d, cores, factors, [target] * d, [0] * d)
    return Workload("exact_recovery", [p], "kron", "fp64", seed)


def decay_problem(rng, n=512, K=32, rmin=8, rmax=32, d=3, basis=128, decay=8.0,
                  target=48, p=10):
    Ps = [haar(rng, n, basis) for _ in range(d)]
    cores, factors = [], []
    for _ in range(K):
        r = rng.integers(rmin, rmax + 1, size=d)
        J = [np.sort(rng.choice(basis, size=int(rk), replace=False)) for rk in r]
        expo = np.zeros(tuple(int(x) for x in r))
        for m in range(d):
            shape = [1] * d
            shape[m] = int(r[m])
            expo = expo + J[m].reshape(shape)
        cores.append(rng.standard_normal(expo.shape) * 10.0 ** (-expo / decay))
        factors.append([Ps[m][:, J[m]] for m in range(d)])
    return Problem([n] * d, cores, factors, [target] * d, [p] * d)


def decay512(seed=20260315, num_problems=1, bf16=True, **kw):
    rng = np.random.default_rng(seed)
    probs = _finish([decay_problem(rng, **kw) for _ in range(num_problems)], bf16)
    return Workload("decay512", probs, "krp", "mixed" if bf16 else "fp64", seed)


def order4(seed=20260316, kind="krp", n=256, K=64, rmin=4, rmax=24, target=40, p=8,
           bf16=True):
    rng = np.random.default_rng(seed)
    d = 4
    cores, factors = [], []
    for k in range(K):
        r = [int(x) for x in rng.integers(rmin, rmax + 1, size=d)]
        cores.append(rng.standard_normal(r) * 2.0 ** (-k / 4))
        factors.append([haar(rng, n, rm) for rm in r])
    probs = _finish([Problem([n] * d, cores, factors, [target] * d, [p] * d)], bf16)
    return Workload("order4", probs, kind, "mixed" if bf16 else "fp64", seed)


def batched(seed=20260317, num_problems=256, bf16=True, p=5):
    rng = np.random.default_rng(seed)
    d = 3
    probs = []
    for _ in range(num_problems):
        n = int(rng.choice([128, 256, 512, 1024]))
        K = int(rng.integers(8, 49))
        ranks = rng.integers(4, 33, size=(K, d))
        med = float(np.median(ranks))
        target = int(np.floor(1.5 * med + 0.5))
        cores = [rng.standard_normal(tuple(int(x) for x in rk)) for rk in ranks]
        factors = [[haar(rng, n, int(x)) for x in rk] for rk in ranks]
        probs.append(Problem([n] * d, cores, factors, [target] * d, [p] * d))
    return Workload("batched", _finish(probs, bf16), "krp", "mixed" if bf16 else "fp64", seed)


def grad384(seed=20260318, n=384, K=16, r=16, target=32, p=8):
    rng = np.random.default_rng(seed)
    d = 3
    cores = [rng.standard_normal((r,) * d) for _ in range(K)]
    factors = [[haar(rng, n, r) for _ in range(d)] for _ in range(K)]
    prob = _finish([Problem([n] * d, cores, factors, [target] * d, [p] * d)], True)
    s = target + p
    T = np.random.default_rng(seed + 1).standard_normal((s,) * d)
    return Workload("grad384", prob, "krp", "mixed", seed, notes=dict(target_tensor=T))


def shared_subspace(seed=20260319, n=200, K=20, d=4, r_true=10, p=2, kind="krp"):
    """Sec. 5.1.1 construction: rank-1 terms in a shared rank-r_true subspace."""
    rng = np.random.default_rng(seed)
    Qs = [haar(rng, n, r_true) for _ in range(d)]
    cores = [np.ones((1,) * d) for _ in range(K)]
    factors = [[Q @ rng.standard_normal((r_true, 1)) for Q in Qs] for _ in range(K)]
    prob = Problem([n] * d, cores, factors, [r_true] * d, [p] * d)
    return Workload("shared_subspace", [prob], kind, "fp64", seed, tol=1e-6)


def cancellation(seed=20260320, n=200, K=60, d=3, r_noise=12, p=2, kind="krp"):
    """Sec. 5.1.2 construction: target plus K/2 noise terms added with + and -."""
    rng = np.random.default_rng(seed)
    diag_t = np.array([1.0, 0.8, 0.6, 2e-6, 1e-6])
    Gt = np.zeros((5,) * d)
    for i, v in enumerate(diag_t):
        Gt[(i,) * d] = v
    Ut = [haar(rng, n, 5) for _ in range(d)]
    diag_n = np.logspace(6, -5, r_noise)
    cores, factors = [], []
    noise = []
    for _ in range(K // 2):
        Gn = np.zeros((r_noise,) * d)
        for i, v in enumerate(diag_n):
            Gn[(i,) * d] = v
        noise.append((Gn, [haar(rng, n, r_noise) for _ in range(d)]))
    for sign in (1.0, -1.0):
        for Gn, Un in noise:
            # X^(i) = X_target / K +- X_noise^(i), each a Tucker term of rank 5 + 12
            G = np.zeros((5 + r_noise,) * d)
            G[(slice(0, 5),) * d] = Gt / K
            G[(slice(5, None),) * d] = sign * Gn
            cores.append(G)
            factors.append([np.hstack([Ut[m], Un[m]]) for m in range(d)])
    prob = Problem([n] * d, cores, factors, [5] * d, [p] * d)
    return Workload("cancellation", [prob], kind, "fp64", seed, tol=1e-6,
                    notes=dict(target_core=Gt, target_factors=Ut))
