"""Python binding of the C ABI in include/tks.h (ctypes; argument marshalling only).

Every step of the method runs in the CUDA kernels of libtks.so; this module only
packs tensors into the documented layouts, passes device pointers and the current
torch CUDA stream, and unpacks results.  There is no fallback: if the library has
not been built, :func:`load` raises.
"""
import ctypes
import os

import numpy as np
import torch

from .build import LIB_PATH

MAX_ORDER = 6
SKETCH = {"kron": 0, "krp": 1}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_f32la": 2}
DTYPE = {"fp64": 0, "bf16": 1}
STATUS = {0: "TKS_OK", 1: "TKS_EINVAL", 2: "TKS_ENOMEM", 3: "TKS_ECUDA", 4: "TKS_ETIMEOUT",
          5: "TKS_ENONFINITE", 6: "TKS_ENOCONV", 7: "TKS_EUNSUPPORTED"}

STEP_KINDS = {0: "omega", 1: "gemm", 2: "reduce", 3: "core_sketch", 4: "qr", 5: "tsqr64", 6: "tc", 7: "simt",
              8: "core_sketch32", 9: "split", 10: "transpose", 11: "qr32", 12: "svd32", 13: "tsqr32",
              14: "core_sketch3", 15: "chain3", 16: "qr_smem32", 17: "project3",
              18: "sketch3", 19: "qr_reg32", 20: "ttm32", 21: "fold4", 22: "project4",
              23: "sketch3f", 24: "sketch4", 25: "svd64", 26: "ttm64", 27: "oz_slice", 28: "oz_gemm", 29: "oz_xmax", 30: "oz_gram", 31: "chol",
              32: "oz_xdig"}


class TksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Problem_t(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("dims", ctypes.POINTER(ctypes.c_int64)),
                ("num_terms", ctypes.c_int32), ("ranks", ctypes.POINTER(ctypes.c_int32)),
                ("target_ranks", ctypes.POINTER(ctypes.c_int32)),
                ("oversampling", ctypes.POINTER(ctypes.c_int32)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("cores", ctypes.c_void_p),
                ("factors", ctypes.POINTER(ctypes.c_void_p))]


class Params_t(ctypes.Structure):
    _fields_ = [("sketch", ctypes.c_int), ("precision", ctypes.c_int), ("dtype", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("trunc_tol", ctypes.c_double), ("omega_lowprec", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("autotune", ctypes.c_int32), ("sketch_qr", ctypes.c_int32),
                ("hosvd_r", ctypes.c_int32), ("proj_chunk", ctypes.c_int32), ("tc_stages", ctypes.c_int32)]

SCHEDULE_KNOBS = ("lanes", "sketch_qr", "hosvd_r", "proj_chunk", "tc_stages")


class PlanInfo_t(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_size_t), ("omega_elems", ctypes.c_int64),
                ("sketch_elems", ctypes.c_int64), ("basis_elems", ctypes.c_int64),
                ("core_elems", ctypes.c_int64), ("output_elems", ctypes.c_int64),
                ("num_problems", ctypes.c_int32), ("launches_recompress", ctypes.c_int32),
                ("flops_lowprec", ctypes.c_double), ("flops_fp64", ctypes.c_double),
                ("grad_core_elems", ctypes.c_int64), ("grad_factor_elems", ctypes.c_int64),
                ("launches_backward", ctypes.c_int32), ("pad", ctypes.c_int32)]


I32x6 = ctypes.c_int32 * MAX_ORDER
I64x6 = ctypes.c_int64 * MAX_ORDER


class ProblemInfo_t(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("R", I32x6), ("omega_cols", I32x6), ("sketch_cols", I32x6),
                ("basis_cols", I32x6), ("max_ranks", I32x6), ("omega_off", I64x6),
                ("sketch_off", I64x6), ("basis_off", I64x6), ("core_off", ctypes.c_int64),
                ("out_core_off", ctypes.c_int64), ("out_factor_off", I64x6),
                ("grad_core_off", ctypes.c_int64), ("grad_factor_off", I64x6)]


class SubrankInfo_t(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_size_t), ("eigenvalue_elems", ctypes.c_int64),
                ("num_problems", ctypes.c_int32), ("launches", ctypes.c_int32), ("max_dim", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("flops", ctypes.c_double)]


class StepProfile_t(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("kind", ctypes.c_int32), ("calls", ctypes.c_int32),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_LIB = None


def load(path=None):
    """Load libtks.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2603_13532_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.tks_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Problem_t), ctypes.c_int32,
                                    ctypes.POINTER(Params_t)]
    lib.tks_plan_destroy.argtypes = [P]
    lib.tks_plan_destroy.restype = None
    lib.tks_plan_info.argtypes = [P, ctypes.POINTER(PlanInfo_t)]
    lib.tks_problem_info.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ProblemInfo_t)]
    I32P = ctypes.POINTER(ctypes.c_int32)
    lib.tks_sketch_sizes.argtypes = [ctypes.c_int32, ctypes.c_int32, I32P, I32P, I32P, I32P]
    lib.tks_sketch_sizes.restype = ctypes.c_int
    lib.tks_generate_omega.argtypes = [P, P, P, P]
    lib.tucker_sum_sketch.argtypes = [P, P, P, P]
    lib.tks_project_core.argtypes = [P, P, P, P, P]
    lib.tucker_sum_recompress.argtypes = [P, P, P, P, P]
    lib.tks_truncate_core.argtypes = [P, P, P, P, P, P, P]
    lib.tks_plan_set_fault_test.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
    lib.tks_project_core_backward.argtypes = [P, P, P, P, P, P, P]
    lib.tks_project_core_backward.restype = ctypes.c_int
    lib.tks_sync_status.argtypes = [P, P]
    lib.tks_plan_tuning.argtypes = [P, ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.tks_truncation_error.argtypes = [P, P, P, P]
    lib.tks_last_error.restype = ctypes.c_char_p
    lib.tks_status_string.restype = ctypes.c_char_p
    lib.tks_status_string.argtypes = [ctypes.c_int]
    lib.tucker_sum_sketch_noalloc.argtypes = [ctypes.POINTER(Problem_t), ctypes.POINTER(Params_t), P, P]
    lib.tucker_sum_sketch_noalloc.restype = ctypes.c_int
    lib.tks_profile_begin.argtypes = [P, ctypes.c_int32]
    lib.tks_profile_end.argtypes = [P, ctypes.POINTER(StepProfile_t), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]
    lib.tks_subrank_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Problem_t), ctypes.c_int32,
                                            ctypes.POINTER(Params_t)]
    lib.tks_subrank_plan_destroy.argtypes = [P]
    lib.tks_subrank_plan_destroy.restype = None
    lib.tks_subrank_info.argtypes = [P, ctypes.POINTER(SubrankInfo_t)]
    lib.tks_subrank_problem_info.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int64)]
    lib.tks_effective_subrank.argtypes = [P, P, P, P, P, P]
    lib.tks_subrank_sync_status.argtypes = [P, P]
    lib.tks_subrank_executed_flops.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    for name in ["tks_plan_create", "tks_plan_info", "tks_problem_info", "tks_generate_omega",
                 "tucker_sum_sketch", "tks_project_core", "tucker_sum_recompress", "tks_sync_status",
                 "tks_profile_begin", "tks_profile_end", "tks_subrank_plan_create", "tks_truncate_core",
                 "tks_plan_set_fault_test", "tks_subrank_info", "tks_plan_tuning", "tks_subrank_executed_flops", "tks_truncation_error",
                 "tks_subrank_problem_info", "tks_effective_subrank", "tks_subrank_sync_status"]:
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(code):
    if code != 0:
        raise TksError(code, _LIB.tks_last_error().decode())


def _stream_handle():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def pack_inputs(problems, dtype, device, pin=False):
    """All problems' inputs in the C-ABI layout inside ONE flat buffer.

    Returns (flat, views) where views[p] = (packed cores, [Ucat_1, ..., Ucat_d]) are views of
    ``flat`` (column-major Ucat_m, cores back to back).  ``device="cpu", pin=True`` builds the
    pinned host staging copy used by the end-to-end measurement.
    """
    tdt = torch.float64 if dtype == "fp64" else torch.bfloat16
    chunks, shapes = [], []
    for prob in problems:
        cores = np.concatenate([np.asarray(G, dtype=np.float64).ravel(order="F") for G in prob.cores])
        parts = [cores]
        for m in range(prob.order):
            Ucat = np.hstack([np.asarray(Us[m], dtype=np.float64) for Us in prob.factors])
            parts.append(Ucat.ravel(order="F"))
        # keep every block 256-byte aligned
        align = 256 // (8 if dtype == "fp64" else 2)
        sizes = []
        for a in parts:
            pad = (-len(a)) % align
            chunks.append(a)
            if pad:
                chunks.append(np.zeros(pad))
            sizes.append(len(a) + pad)
        shapes.append(sizes)
    host = torch.from_numpy(np.concatenate(chunks)).to(tdt)
    flat = host.pin_memory() if pin else host.to(device)
    views, off = [], 0
    for prob, sizes in zip(problems, shapes):
        v = []
        for sz in sizes:
            v.append(flat[off: off + sz])
            off += sz
        views.append((v[0], v[1:]))
    return flat, views


def _problem_structs(problems, inputs, keep):
    """tks_problem array over ``problems`` with device inputs ``inputs`` (from pack_inputs); the
    host arrays it points to are appended to ``keep`` and must outlive the C call."""
    arr = (Problem_t * len(problems))()
    for i, (p, (core_t, facs)) in enumerate(zip(problems, inputs)):
        d = p.order
        dims = (ctypes.c_int64 * d)(*p.dims)
        ranks = (ctypes.c_int32 * (p.num_terms * d))(*[r for rk in p.ranks() for r in rk])
        tgt = (ctypes.c_int32 * d)(*p.target)
        ovs = (ctypes.c_int32 * d)(*p.oversampling)
        alpha = (ctypes.c_double * p.num_terms)(*p.alpha) if p.alpha is not None else None
        fptrs = (ctypes.c_void_p * d)(*[f.data_ptr() for f in facs])
        keep += [dims, ranks, tgt, ovs, alpha, fptrs]
        arr[i] = Problem_t(d, dims, p.num_terms, ranks, tgt, ovs,
                           ctypes.cast(alpha, ctypes.POINTER(ctypes.c_double)) if alpha else None,
                           ctypes.c_void_p(core_t.data_ptr()), fptrs)
    return arr


class Plan:
    """A plan over a list of ``workloads.Problem`` with their device inputs."""

    def __init__(self, problems, kind="krp", precision="fp64", seed=0, tol=0.0, device="cuda", omega_lowprec=False,
                 lanes=0, autotune=False, schedule=None):
        """``schedule``: a dict of tks_params schedule knobs (the "picked" object of tuning()), which
        overrides ``lanes``; ``autotune``: let tks_plan_create search them on these inputs."""
        self.lib = load()
        self.problems = list(problems)
        self.kind, self.precision, self.seed, self.tol = kind, precision, seed, tol
        self.dtype = "fp64" if precision == "fp64" else "bf16"
        self.device = torch.device(device)
        self.flat_inputs, self.inputs = pack_inputs(self.problems, self.dtype, self.device)
        self._keep = []
        arr = _problem_structs(self.problems, self.inputs, self._keep)
        prm = Params_t(SKETCH[kind], PRECISION[precision], DTYPE[self.dtype], seed, tol, int(omega_lowprec), int(lanes))
        for k, v in (schedule or {}).items():
            if k not in SCHEDULE_KNOBS:
                raise ValueError(f"unknown schedule knob {k}")
            setattr(prm, k, int(v))
        prm.autotune = int(bool(autotune))
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.tks_plan_create(ctypes.byref(handle), arr, len(self.problems), ctypes.byref(prm)))
        self.handle = handle
        self.info = PlanInfo_t()
        _check(self.lib.tks_plan_info(handle, ctypes.byref(self.info)))
        self.pinfo = []
        for i in range(len(self.problems)):
            pi = ProblemInfo_t()
            _check(self.lib.tks_problem_info(handle, i, ctypes.byref(pi)))
            self.pinfo.append(pi)
        self.workspace = torch.empty(max(1, self.info.workspace_bytes), dtype=torch.uint8, device=self.device)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.tks_plan_destroy(h)
            self.handle = None

    def truncation_error(self):
        """||H - H~|| / ||H|| of every problem's last ST-HOSVD (tks_truncation_error), as a numpy array."""
        out = torch.zeros(max(1, len(self.problems)), dtype=torch.float64, device=self.device)
        _check(self.lib.tks_truncation_error(self.handle, _ptr(self.workspace), _ptr(out), _stream_handle()))
        self.sync()
        return out[: len(self.problems)].cpu().numpy()

    def tuning(self):
        """The schedule the plan runs and, when autotuned, the candidates timed (tks_plan_tuning)."""
        import json
        n = ctypes.c_int64()
        _check(self.lib.tks_plan_tuning(self.handle, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(self.lib.tks_plan_tuning(self.handle, buf, n.value + 1, ctypes.byref(n)))
        return json.loads(buf.value.decode())

    # ---- raw entry points (device buffers in, nothing synchronised)
    def omega_raw(self, out):
        _check(self.lib.tks_generate_omega(self.handle, _ptr(self.workspace), _ptr(out), _stream_handle()))

    def sketch_raw(self, Y):
        _check(self.lib.tucker_sum_sketch(self.handle, _ptr(self.workspace), _ptr(Y), _stream_handle()))

    def project_raw(self, Q, H):
        _check(self.lib.tks_project_core(self.handle, _ptr(self.workspace), _ptr(Q), _ptr(H), _stream_handle()))

    def backward_raw(self, Q, Hbar, dcores, dfactors):
        _check(self.lib.tks_project_core_backward(self.handle, _ptr(self.workspace), _ptr(Q), _ptr(Hbar),
                                                  _ptr(dcores), _ptr(dfactors), _stream_handle()))

    def truncate_raw(self, Q, H, out, ranks):
        _check(self.lib.tks_truncate_core(self.handle, _ptr(self.workspace), _ptr(Q), _ptr(H), _ptr(out), _ptr(ranks),
                                          _stream_handle()))

    def recompress_raw(self, out, ranks):
        _check(self.lib.tucker_sum_recompress(self.handle, _ptr(self.workspace), _ptr(out), _ptr(ranks),
                                              _stream_handle()))

    def set_fault_test(self, wait_cycles=0, stall=False):
        _check(self.lib.tks_plan_set_fault_test(self.handle, int(wait_cycles), int(stall)))

    def sync(self):
        _check(self.lib.tks_sync_status(self.handle, _stream_handle()))

    def profile_begin(self, max_calls):
        _check(self.lib.tks_profile_begin(self.handle, max_calls))

    def profile_end(self):
        """Stage timings of the recompress calls since profile_begin: one dict per launch."""
        n = ctypes.c_int32()
        arr = (StepProfile_t * 512)()
        _check(self.lib.tks_profile_end(self.handle, arr, 512, ctypes.byref(n)))
        return [dict(name=a.name.decode(), kind=STEP_KINDS.get(a.kind, a.kind), calls=a.calls, ms=a.ms,
                     flops=a.flops, bytes=a.bytes) for a in arr[:min(n.value, 512)]]

    # ---- convenience: allocate, run, return numpy per problem
    def _new(self, n, dtype=torch.float64):
        return torch.zeros(max(1, n), dtype=dtype, device=self.device)

    def omega(self):
        out = self._new(self.info.omega_elems)
        self.omega_raw(out)
        self.sync()
        host = out.cpu().numpy()
        res = []
        for p, pi in zip(self.problems, self.pinfo):
            res.append([host[pi.omega_off[m]: pi.omega_off[m] + p.dims[m] * pi.omega_cols[m]]
                        .reshape(p.dims[m], pi.omega_cols[m], order="F") for m in range(p.order)])
        return res

    def sketch(self):
        Y = self._new(self.info.sketch_elems)
        self.sketch_raw(Y)
        self.sync()
        host = Y.cpu().numpy()
        return [[host[pi.sketch_off[m]: pi.sketch_off[m] + p.dims[m] * pi.sketch_cols[m]]
                 .reshape(p.dims[m], pi.sketch_cols[m], order="F") for m in range(p.order)]
                for p, pi in zip(self.problems, self.pinfo)]

    def pack_bases(self, Qs):
        host = np.zeros(max(1, self.info.basis_elems))
        for p, pi, Qp in zip(self.problems, self.pinfo, Qs):
            for m in range(p.order):
                b = pi.basis_cols[m]
                host[pi.basis_off[m]: pi.basis_off[m] + p.dims[m] * b] = np.asarray(Qp[m])[:, :b].ravel(order="F")
        return torch.from_numpy(host).to(self.device)

    def project(self, Qs):
        Q = self.pack_bases(Qs)
        H = self._new(self.info.core_elems)
        self.project_raw(Q, H)
        self.sync()
        host = H.cpu().numpy()
        out = []
        for p, pi in zip(self.problems, self.pinfo):
            shape = [pi.basis_cols[m] for m in range(p.order)]
            out.append(host[pi.core_off: pi.core_off + int(np.prod(shape))].reshape(shape, order="F"))
        return out

    def pack_core(self, Hs):
        host = np.zeros(max(1, self.info.core_elems))
        for p, pi, H in zip(self.problems, self.pinfo, Hs):
            H = np.asarray(H)
            host[pi.core_off: pi.core_off + H.size] = H.ravel(order="F")
        return torch.from_numpy(host).to(self.device)

    def backward(self, Qs, Hbars):
        """dL/dG_k and dL/dU_k^(n) (lists per problem) for dL/dH = Hbars, bases Qs held fixed."""
        Q = self.pack_bases(Qs)
        Hb = self.pack_core(Hbars)
        dc = self._new(self.info.grad_core_elems)
        df = self._new(self.info.grad_factor_elems)
        self.backward_raw(Q, Hb, dc, df)
        self.sync()
        dc, df = dc.cpu().numpy(), df.cpu().numpy()
        res = []
        for p, pi in zip(self.problems, self.pinfo):
            dG, off = [], pi.grad_core_off
            for G in p.cores:
                dG.append(dc[off: off + G.size].reshape(G.shape, order="F"))
                off += G.size
            dU = []
            for m in range(p.order):
                R = pi.R[m]
                Ucat = df[pi.grad_factor_off[m]: pi.grad_factor_off[m] + p.dims[m] * R].reshape(p.dims[m], R,
                                                                                                order="F")
                cols, c0 = [], 0
                for G in p.cores:
                    cols.append(Ucat[:, c0: c0 + G.shape[m]])
                    c0 += G.shape[m]
                dU.append(cols)
            res.append((dG, [[dU[m][k] for m in range(p.order)] for k in range(p.num_terms)]))
        return res

    def recompress(self):
        out = self._new(self.info.output_elems)
        ranks = torch.zeros(len(self.problems) * MAX_ORDER, dtype=torch.int32, device=self.device)
        self.recompress_raw(out, ranks)
        self.sync()
        return self.unpack(out, ranks)

    def truncate(self, Qs, Hs):
        """The ST-HOSVD truncation alone of given bases Qs and projected cores Hs (lists per problem)."""
        Q = self.pack_bases(Qs)
        H = self.pack_core(Hs)
        out = self._new(self.info.output_elems)
        ranks = torch.zeros(len(self.problems) * MAX_ORDER, dtype=torch.int32, device=self.device)
        self.truncate_raw(Q, H, out, ranks)
        self.sync()
        return self.unpack(out, ranks)

    def unpack(self, out, ranks):
        host = out.cpu().numpy()
        rk = ranks.cpu().numpy().reshape(-1, MAX_ORDER)
        res = []
        for i, (p, pi) in enumerate(zip(self.problems, self.pinfo)):
            rmax = [pi.max_ranks[m] for m in range(p.order)]
            core = host[pi.out_core_off: pi.out_core_off + int(np.prod(rmax))].reshape(rmax, order="F")
            facs = [host[pi.out_factor_off[m]: pi.out_factor_off[m] + p.dims[m] * rmax[m]]
                    .reshape(p.dims[m], rmax[m], order="F") for m in range(p.order)]
            res.append(dict(core=core, factors=facs, ranks=[int(x) for x in rk[i, :p.order]]))
        return res


class ProjectCore(torch.autograd.Function):
    """H(G, U; Q) = sum_k alpha_k G_k x_1 (Q_1^T U_k^(1)) ... x_d (Q_d^T U_k^(d)) as an autograd op.

    Differentiable input: ``plan.flat_inputs`` (the plan's packed cores and factors; the plan reads
    them in place).  Q is a constant: its gradient is not computed (stop-gradient), matching a
    method whose bases come from a QR that is not differentiated.  Forward and backward both run
    in libtks.so (tks_project_core / tks_project_core_backward); the backward recomputes
    A_kn = Q_n^T U_k^(n) instead of storing it.
    """

    @staticmethod
    def forward(ctx, flat_inputs, Q, plan):
        H = torch.zeros(max(1, plan.info.core_elems), dtype=torch.float64, device=plan.device)
        plan.project_raw(Q, H)
        ctx.plan = plan
        ctx.save_for_backward(Q)
        ctx.mark_non_differentiable(Q)
        return H

    @staticmethod
    def backward(ctx, gH):
        (Q,) = ctx.saved_tensors
        plan = ctx.plan
        gH = gH.contiguous().to(torch.float64)
        dc = torch.zeros(max(1, plan.info.grad_core_elems), dtype=torch.float64, device=plan.device)
        df = torch.zeros(max(1, plan.info.grad_factor_elems), dtype=torch.float64, device=plan.device)
        plan.backward_raw(Q, gH, dc, df)
        grad = torch.zeros_like(plan.flat_inputs)
        base = plan.flat_inputs.storage_offset()
        for p, pi, (core_v, fac_v) in zip(plan.problems, plan.pinfo, plan.inputs):
            nc = sum(G.size for G in p.cores)
            o = core_v.storage_offset() - base
            grad[o: o + nc] = dc[pi.grad_core_off: pi.grad_core_off + nc]
            for m in range(p.order):
                nf = p.dims[m] * pi.R[m]
                o = fac_v[m].storage_offset() - base
                grad[o: o + nf] = df[pi.grad_factor_off[m]: pi.grad_factor_off[m] + nf]
        return grad, None, None


class SubrankPlan:
    """The effective subrank heuristic (Alg. 5) over a list of ``workloads.Problem``.

    ``eps`` is the user tolerance; each problem's ``oversampling`` gives p_n (its ``target`` is
    not used).  ``dtype`` is the element type the inputs are passed in ("fp64" or "bf16").
    """

    def __init__(self, problems, eps, dtype="fp64", device="cuda", inputs=None):
        self.lib = load()
        self.problems = list(problems)
        self.eps, self.dtype = eps, dtype
        self.device = torch.device(device)
        if inputs is None:
            self.flat_inputs, self.inputs = pack_inputs(self.problems, dtype, self.device)
        else:
            self.inputs = inputs
        self._keep = []
        arr = _problem_structs(self.problems, self.inputs, self._keep)
        prm = Params_t(SKETCH["krp"], PRECISION["fp64"], DTYPE[dtype], 0, float(eps), 0, 0)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.tks_subrank_plan_create(ctypes.byref(handle), arr, len(self.problems), ctypes.byref(prm)))
        self.handle = handle
        self.info = SubrankInfo_t()
        _check(self.lib.tks_subrank_info(handle, ctypes.byref(self.info)))
        self.dims, self.eig_off = [], []
        for i in range(len(self.problems)):
            dims = (ctypes.c_int32 * MAX_ORDER)()
            offs = (ctypes.c_int64 * MAX_ORDER)()
            _check(self.lib.tks_subrank_problem_info(handle, i, dims, offs))
            self.dims.append(list(dims))
            self.eig_off.append(list(offs))
        self.workspace = torch.empty(max(1, self.info.workspace_bytes), dtype=torch.uint8, device=self.device)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.tks_subrank_plan_destroy(h)
            self.handle = None

    def run_raw(self, ranks, ell, evals=None):
        _check(self.lib.tks_effective_subrank(self.handle, _ptr(self.workspace), _ptr(ranks), _ptr(ell),
                                              _ptr(evals) if evals is not None else None, _stream_handle()))

    def set_fault_test(self, wait_cycles=0, stall=False):
        _check(self.lib.tks_plan_set_fault_test(self.handle, int(wait_cycles), int(stall)))

    def sync(self):
        _check(self.lib.tks_subrank_sync_status(self.handle, _stream_handle()))

    def executed_flops(self):
        """Flops the last run executed (Gram matrices plus the reduction steps before the early end)."""
        f = ctypes.c_double()
        _check(self.lib.tks_subrank_executed_flops(self.handle, ctypes.byref(f)))
        return f.value

    def run(self, eigenvalues=False):
        """Per problem: dict(rank=[rank_n], ell=[ell_n], lam=[descending eigenvalues] or None)."""
        n = len(self.problems) * MAX_ORDER
        ranks = torch.zeros(n, dtype=torch.int32, device=self.device)
        ell = torch.zeros(n, dtype=torch.int32, device=self.device)
        ev = torch.zeros(max(1, self.info.eigenvalue_elems), dtype=torch.float64, device=self.device) \
            if eigenvalues else None
        self.run_raw(ranks, ell, ev)
        self.sync()
        rk = ranks.cpu().numpy().reshape(-1, MAX_ORDER)
        el = ell.cpu().numpy().reshape(-1, MAX_ORDER)
        host = ev.cpu().numpy() if eigenvalues else None
        res = []
        for i, p in enumerate(self.problems):
            lam = None
            if eigenvalues:
                lam = [host[self.eig_off[i][m]: self.eig_off[i][m] + self.dims[i][m]] for m in range(p.order)]
            res.append(dict(rank=[int(x) for x in rk[i, :p.order]], ell=[int(x) for x in el[i, :p.order]],
                            lam=lam))
        return res


def with_sketch_ranks(problems, ells):
    """Copies of ``problems`` whose plan sketches with ell_n from the subrank heuristic: target_n =
    ell_n and oversampling 0 (so a Plan with ``tol=eps`` runs Alg. 3/4 as printed, the final
    ST-HOSVD ranks capped at ell_n)."""
    import dataclasses
    return [dataclasses.replace(p, target=list(e), oversampling=[0] * p.order) for p, e in zip(problems, ells)]


def sketch_sizes(kind, target, oversampling):
    """(columns of Omega_m, columns S_m of Y_m) per mode, from tks_sketch_sizes (host-only: no plan
    and no device)."""
    lib = load()
    d = len(target)
    arr = ctypes.c_int32 * d
    cols, S = arr(), arr()
    _check(lib.tks_sketch_sizes(SKETCH[kind], d, arr(*target), arr(*oversampling), cols, S))
    return list(cols), list(S)
