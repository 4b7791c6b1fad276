"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/tks.h
declares, and rejects invalid arguments before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tks.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2603_13532_gb300 import binding, build
    build.build()
    return binding.load()


def declared_symbols():
    names = []
    for line in open(HEADER):
        m = re.match(r"TKS_API\s+[\w\s\*]*?\b(\w+)\s*\(", line)
        if m:
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for name in ["tks_plan_create", "tucker_sum_sketch", "tucker_sum_recompress", "tks_project_core",
                 "tks_generate_omega", "tks_sync_status", "tks_plan_destroy"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2603_13532_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_library_has_no_cuda_runtime_dependency(lib):
    from paper_2603_13532_gb300 import build
    out = subprocess.run(["ldd", build.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcudart" not in out


def _problem(binding, dims=(5, 6, 7), ranks=((2, 2, 2),), target=(3, 3, 3), over=(1, 1, 1)):
    d = len(dims)
    keep = dict(
        dims=(ctypes.c_int64 * d)(*dims),
        ranks=(ctypes.c_int32 * (len(ranks) * d))(*[r for rk in ranks for r in rk]),
        tgt=(ctypes.c_int32 * d)(*target),
        ovs=(ctypes.c_int32 * d)(*over),
        facs=(ctypes.c_void_p * d)(*([0x1000] * d)),
    )
    p = binding.Problem_t(d, keep["dims"], len(ranks), keep["ranks"], keep["tgt"], keep["ovs"], None,
                          ctypes.c_void_p(0x1000), keep["facs"])
    return p, keep


@pytest.mark.parametrize("mutate,code", [
    (lambda p, k: setattr(p, "order", 1), 1),
    (lambda p, k: setattr(p, "num_terms", 0), 1),
    (lambda p, k: setattr(p, "num_terms", 2 ** 20 + 1), 1),   # rejected before the ranks are read
    (lambda p, k: k["ranks"].__setitem__(0, 0), 1),
    (lambda p, k: k["ranks"].__setitem__(1, 65), 1),
    (lambda p, k: k["ranks"].__setitem__(0, 6), 1),     # rank above n_1 = 5
    (lambda p, k: k["tgt"].__setitem__(2, 0), 1),
    (lambda p, k: k["ovs"].__setitem__(0, -1), 1),
    (lambda p, k: k["ovs"].__setitem__(1, 2 ** 31 - 4), 1),   # ell above 2^21 (and above INT32_MAX)
    (lambda p, k: setattr(p, "cores", None), 1),
    (lambda p, k: k["tgt"].__setitem__(0, 200), 7),      # basis b = min(n, S) = 201 > TKS_MAX_BASIS
])
def test_plan_create_rejects_bad_problems(lib, mutate, code):
    from paper_2603_13532_gb300 import binding
    p, keep = _problem(binding, dims=(500, 6, 7) if code == 7 else (5, 6, 7))
    mutate(p, keep)
    prm = binding.Params_t(1, 0, 0, 1, 0.0)
    h = ctypes.c_void_p()
    rc = lib.tks_plan_create(ctypes.byref(h), ctypes.byref(p), 1, ctypes.byref(prm))
    assert rc == code, lib.tks_last_error()
    assert not h.value
    assert lib.tks_last_error()


def test_plan_create_rejects_bad_params(lib):
    from paper_2603_13532_gb300 import binding
    p, keep = _problem(binding)
    h = ctypes.c_void_p()
    for prm in [binding.Params_t(5, 0, 0, 1, 0.0), binding.Params_t(1, 0, 1, 1, 0.0),
                binding.Params_t(1, 0, 0, 1, -1.0), binding.Params_t(1, 9, 0, 1, 0.0),
                binding.Params_t(1, 0, 0, 1, 0.0, 2), binding.Params_t(1, 0, 0, 1, 0.0, 0, 9),
                binding.Params_t(1, 0, 0, 1, 0.0, 0, -1)]:
        assert lib.tks_plan_create(ctypes.byref(h), ctypes.byref(p), 1, ctypes.byref(prm)) == 1
    assert lib.tks_plan_create(None, ctypes.byref(p), 1, ctypes.byref(binding.Params_t(1, 0, 0, 1, 0.0))) == 1
    assert lib.tks_plan_create(ctypes.byref(h), ctypes.byref(p), 0, ctypes.byref(binding.Params_t(1, 0, 0, 1, 0.0))) == 1
    # more than 2^20 problems: rejected before any problem is read
    assert lib.tks_plan_create(ctypes.byref(h), ctypes.byref(p), 2 ** 20 + 1,
                               ctypes.byref(binding.Params_t(1, 0, 0, 1, 0.0))) == 1


def test_execute_rejects_null_plan(lib):
    for f in (lib.tucker_sum_sketch, lib.tks_generate_omega):
        assert f(None, None, None, None) == 1
    assert lib.tucker_sum_recompress(None, None, None, None, None) == 1
    assert lib.tks_project_core(None, None, None, None, None) == 1
    assert lib.tks_plan_info(None, None) == 1


def test_status_strings(lib):
    assert lib.tks_status_string(0) == b"TKS_OK"
    assert lib.tks_status_string(6) == b"TKS_ENOCONV"


@pytest.mark.parametrize("mutate,eps,code", [
    (lambda p, k: None, 0.0, 1),                          # the heuristic needs eps > 0
    (lambda p, k: None, float("nan"), 1),
    (lambda p, k: setattr(p, "order", 7), 1e-6, 1),
    (lambda p, k: k["ranks"].__setitem__(2, 0), 1e-6, 1),
    (lambda p, k: k["ovs"].__setitem__(1, -2), 1e-6, 1),
    (lambda p, k: setattr(p, "cores", None), 1e-6, 1),
])
def test_subrank_plan_rejects_bad_arguments(lib, mutate, eps, code):
    from paper_2603_13532_gb300 import binding
    p, keep = _problem(binding)
    mutate(p, keep)
    prm = binding.Params_t(1, 0, 0, 1, eps)
    h = ctypes.c_void_p()
    assert lib.tks_subrank_plan_create(ctypes.byref(h), ctypes.byref(p), 1, ctypes.byref(prm)) == code
    assert not h.value
    assert lib.tks_last_error()


def test_subrank_plan_rejects_oversized_gram(lib):
    # min(n, R) = min(3000, 47 x 64) = 3000 > 2048: unsupported, reported before any device call
    from paper_2603_13532_gb300 import binding
    p, keep = _problem(binding, dims=(3000, 64, 64), ranks=tuple((64, 2, 2) for _ in range(47)))
    h = ctypes.c_void_p()
    prm = binding.Params_t(1, 0, 0, 1, 1e-6)
    assert lib.tks_subrank_plan_create(ctypes.byref(h), ctypes.byref(p), 1, ctypes.byref(prm)) == 7
    assert b"2048" in lib.tks_last_error()


def test_subrank_execute_rejects_null_arguments(lib):
    assert lib.tks_effective_subrank(None, None, None, None, None, None) == 1
    assert lib.tks_subrank_info(None, None) == 1
    assert lib.tks_subrank_sync_status(None, None) == 1
