"""ctypes binding of ``libccs.so`` (``include/ccs.h``), same names as the C ABI.

Argument marshalling only: circuits, cuts and options are packed into the
C structs, device memory comes from torch's caching allocator through the
``ccs_allocator`` callbacks, and work is issued on torch's current CUDA
stream.  Every step of the path runs in the library's kernels; there is no
Python or CPU fallback, and a missing library or GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccs.so")

CCS_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED_GATE", -3: "TOO_MANY_CUTS", -4: "NC_TOO_WIDE",
          -5: "OOM", -6: "CUDA", -7: "TIMEOUT", -8: "UNSUPPORTED", -9: "DEVICE_CHECK"}
CCS_EXACT, CCS_SAMPLED, CCS_STITCH = 0, 1, 2
CCS_FP32, CCS_BF16 = 0, 1
CCS_ML_SAMPLED, CCS_ML_ALL = 0, 1

# Every symbol include/ccs.h declares (checked by the ABI test).
EXPORTS = ["ccs_version", "ccs_create", "ccs_destroy", "ccs_last_error", "ccs_build_fragments",
           "ccs_plan_free", "ccs_eval_variants", "ccs_res_free", "ccs_recombine", "ccs_plan_counts",
           "ccs_fragment_info_get", "ccs_plan_cuts", "ccs_fragment_wires", "ccs_get_tableau",
           "ccs_get_outcome_space", "ccs_get_counts", "ccs_get_dist", "ccs_get_zvals", "ccs_get_tensor",
           "ccs_set_profiling", "ccs_get_stage_times", "ccs_cut_candidates", "ccs_recombine_noalloc",
           "ccs_get_tuning", "ccs_get_operand", "ccs_launch_count", "ccs_ml_correct"]
STAGES = ["clifford", "sample", "statevector", "fold", "recombine", "operands"]


class ccs_gate(C.Structure):
    _fields_ = [("op", C.c_uint8), ("nq", C.c_uint8), ("flags", C.c_uint16),
                ("q", C.c_uint32 * 2), ("param", C.c_double)]


# numpy twin of ccs_gate (same offsets), for packing whole circuits at once
_GATE_DTYPE = np.dtype({"names": ["op", "nq", "flags", "q", "param"],
                        "formats": [np.uint8, np.uint8, np.uint16, (np.uint32, 2), np.float64],
                        "offsets": [ccs_gate.op.offset, ccs_gate.nq.offset, ccs_gate.flags.offset,
                                    ccs_gate.q.offset, ccs_gate.param.offset],
                        "itemsize": C.sizeof(ccs_gate)})


class ccs_cut(C.Structure):
    _fields_ = [("qubit", C.c_uint32), ("gate_index", C.c_uint32)]


class ccs_problem(C.Structure):
    _fields_ = [("n_qubits", C.c_uint32), ("n_gates", C.c_uint32), ("gates", C.POINTER(ccs_gate)),
                ("n_cuts", C.c_int32), ("cuts", C.POINTER(ccs_cut)),
                ("n_marginal", C.c_uint32), ("marginal", C.POINTER(C.c_uint32)),
                ("n_zstrings", C.c_uint32), ("zstring_offsets", C.POINTER(C.c_uint32)),
                ("zstring_qubits", C.POINTER(C.c_uint32))]


class ccs_cut_opts(C.Structure):
    _fields_ = [("max_cuts", C.c_int32), ("max_nc_width", C.c_int32), ("use_learned", C.c_int32)]


class ccs_eval_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("shots", C.c_uint32), ("seed_lo", C.c_uint32),
                ("seed_hi", C.c_uint32), ("keep_tableaus", C.c_int32), ("use_graph", C.c_int32),
                ("autotune", C.c_int32), ("per_variant_body", C.c_int32), ("hub_sampler", C.c_int32)]


class ccs_recomb_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("outputs_on_device", C.c_int32), ("no_tensor_cores", C.c_int32),
                ("use_graph", C.c_int32), ("k_lo", C.c_uint64), ("k_hi", C.c_uint64)]


class ccs_fragment_info(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("n_wires", "clifford", "n_variants", "n_qin", "n_qout",
                                           "n_marg", "n_meas", "n_slots", "n_ops", "n_moments",
                                           "n_zstrings")]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class ccs_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class CCSError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libccs.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is None:
        from . import build as _build
        _build.build()
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "ccs_version": ([], C.c_char_p),
            "ccs_create": ([C.POINTER(P), C.c_int, P, C.POINTER(ccs_allocator)], C.c_int),
            "ccs_destroy": ([P], None),
            "ccs_last_error": ([P], C.c_char_p),
            "ccs_build_fragments": ([P, C.POINTER(ccs_problem), C.c_int, C.POINTER(ccs_cut_opts),
                                     C.POINTER(P)], C.c_int),
            "ccs_plan_free": ([P], None),
            "ccs_eval_variants": ([P, P, C.POINTER(ccs_eval_opts), C.POINTER(P)], C.c_int),
            "ccs_res_free": ([P], None),
            "ccs_recombine": ([P, P, P, C.POINTER(ccs_recomb_opts), P, P], C.c_int),
            "ccs_plan_counts": ([P, P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
            "ccs_fragment_info_get": ([P, P, C.c_int, C.c_int, C.POINTER(ccs_fragment_info)], C.c_int),
            "ccs_plan_cuts": ([P, P, C.c_int, C.POINTER(ccs_cut), C.c_int], C.c_int),
            "ccs_fragment_wires": ([P, P, C.c_int, C.c_int, C.POINTER(C.c_uint32)], C.c_int),
            "ccs_get_tableau": ([P, P, C.c_int, C.c_int, C.c_int, P], C.c_int),
            "ccs_get_outcome_space": ([P, P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64), C.POINTER(C.c_int)], C.c_int),
            "ccs_get_counts": ([P, P, C.c_int, C.c_int, C.c_int, P], C.c_int),
            "ccs_get_dist": ([P, P, C.c_int, C.c_int, C.c_int, P], C.c_int),
            "ccs_get_zvals": ([P, P, C.c_int, C.c_int, C.c_int, P], C.c_int),
            "ccs_get_tensor": ([P, P, C.c_int, C.c_int, P], C.c_int),
            "ccs_get_operand": ([P, P, C.c_int, C.c_int, P], C.c_int),
            "ccs_set_profiling": ([P, C.c_int], C.c_int),
            "ccs_recombine_noalloc": ([P, P, P, C.c_int, P, P], C.c_int),
            "ccs_ml_correct": ([P, P, P, C.c_int], C.c_int),
            "ccs_get_tuning": ([P, P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
            "ccs_cut_candidates": ([P, C.POINTER(ccs_problem), C.POINTER(ccs_cut_opts), C.POINTER(ccs_cut),
                                    C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int], C.c_int),
            "ccs_get_stage_times": ([P, C.POINTER(C.c_double), C.c_int], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class _TorchAllocator:
    """Device memory from torch's caching allocator, kept alive by pointer."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.blocks = {}
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)
        self.struct = ccs_allocator(self.c_alloc, self.c_free, None)

    def _alloc(self, nbytes, stream, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.blocks[p] = t
        return p

    def _free(self, ptr, nbytes, stream, user):
        self.blocks.pop(ptr, None)


class Ctx:
    def __init__(self, handle, allocator, stream):
        self.h = handle
        self.allocator = allocator
        self.stream = stream

    def check(self, rc, what):
        if rc < 0:
            msg = lib().ccs_last_error(self.h).decode()
            raise CCSError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")
        return rc

    def close(self):
        if self.h:
            lib().ccs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    def __init__(self, ctx, handle, problems):
        self.ctx, self.h, self.problems = ctx, handle, problems

    def __del__(self):
        try:
            if self.h:
                lib().ccs_plan_free(self.h)
        except Exception:
            pass


class Res:
    def __init__(self, ctx, plan, handle):
        self.ctx, self.plan, self.h = ctx, plan, handle

    def __del__(self):
        try:
            if self.h:
                lib().ccs_res_free(self.h)
        except Exception:
            pass


def ccs_version():
    return lib().ccs_version().decode()


def ccs_create(device=0, torch_allocator=True):
    """Context on ``device`` using torch's current stream (and allocator).

    ``device=-1`` gives a host-only context for building and inspecting plans."""
    if device < 0:
        h = C.c_void_p()
        rc = lib().ccs_create(C.byref(h), -1, None, None)
        if rc != CCS_OK:
            raise CCSError(f"ccs_create failed: {ERRORS.get(rc, rc)}")
        return Ctx(h, None, None)
    import torch
    if not torch.cuda.is_available():
        raise CCSError("no CUDA device: the circuit-cutting path runs only on the GPU")
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    alloc = _TorchAllocator(torch.device("cuda", device)) if torch_allocator else None
    h = C.c_void_p()
    rc = lib().ccs_create(C.byref(h), device, C.c_void_p(stream.cuda_stream),
                          C.byref(alloc.struct) if alloc else None)
    if rc != CCS_OK:
        raise CCSError(f"ccs_create failed: {ERRORS.get(rc, rc)}")
    return Ctx(h, alloc, stream)


def _pack_problem(prob):
    """prob: object with .circuit (n_qubits, gates=[(op,q0,q1)] or
    (10, q, -1, a) for Z^a), .cuts (or None), .marginal, .zstrings."""
    circ = prob.circuit
    ng = len(circ.gates)
    arr = np.zeros(max(1, ng), dtype=_GATE_DTYPE)
    if ng:
        g = np.asarray([t[:3] for t in circ.gates], dtype=np.int64).reshape(ng, 3)
        arr["op"][:ng] = g[:, 0]
        arr["q"][:ng, 0] = g[:, 1]
        arr["q"][:ng, 1] = np.maximum(g[:, 2], 0)
        zp = [(i, t[3]) for i, t in enumerate(circ.gates) if len(t) > 3]
        if zp:
            idx, val = zip(*zp)
            arr["param"][list(idx)] = val
    gates = (ccs_gate * max(1, ng)).from_buffer(arr)
    cuts = getattr(prob, "cuts", None)
    ccuts = (ccs_cut * max(1, len(cuts) if cuts else 1))()
    if cuts:
        for i, (q, g) in enumerate(cuts):
            ccuts[i].qubit, ccuts[i].gate_index = q, g
    marg = (C.c_uint32 * max(1, len(prob.marginal)))(*prob.marginal)
    zs = list(getattr(prob, "zstrings", []) or [])
    offs = [0]
    flat = []
    for z in zs:
        flat += list(z)
        offs.append(len(flat))
    zo = (C.c_uint32 * len(offs))(*offs)
    zq = (C.c_uint32 * max(1, len(flat)))(*flat)
    p = ccs_problem(circ.n_qubits, len(circ.gates), gates, -1 if cuts is None else len(cuts), ccuts,
                    len(prob.marginal), marg, len(zs), zo, zq)
    keep = (arr, gates, ccuts, marg, zo, zq)
    return p, keep


class PackedProblems:
    """Problems marshalled once into ccs_problem structs (host buffers the
    C ABI reads); pass to ccs_build_fragments in place of the list."""

    def __init__(self, problems):
        self.problems = list(problems)
        self._keep = [_pack_problem(p) for p in self.problems]
        self.arr = (ccs_problem * len(self._keep))(*[p for p, _ in self._keep])

    def __len__(self):
        return len(self.problems)


def pack_problems(problems):
    return PackedProblems(problems)


def ccs_build_fragments(ctx, problems, max_cuts=12, max_nc_width=10, use_learned=0):
    pk = problems if isinstance(problems, PackedProblems) else PackedProblems(problems)
    opts = ccs_cut_opts(max_cuts, max_nc_width, use_learned)
    h = C.c_void_p()
    ctx.check(lib().ccs_build_fragments(ctx.h, pk.arr, len(pk), C.byref(opts), C.byref(h)),
              "ccs_build_fragments")
    return Plan(ctx, h, pk.problems)


def ccs_eval_variants(ctx, plan, mode=CCS_SAMPLED, shots=1024, seed_lo=0x1234, seed_hi=0x5678,
                      keep_tableaus=False, use_graph=False, res=None, autotune=False, per_variant_body=False,
                      hub_sampler=0):
    opts = ccs_eval_opts(mode, shots, seed_lo, seed_hi, int(keep_tableaus), int(use_graph), int(autotune),
                         int(per_variant_body), int(hub_sampler))
    h = C.c_void_p(res.h.value if res is not None else None)
    ctx.check(lib().ccs_eval_variants(ctx.h, plan.h, C.byref(opts), C.byref(h)), "ccs_eval_variants")
    if res is not None:
        return res
    return Res(ctx, plan, h)


def ccs_recombine(ctx, plan, res, precision=CCS_FP32, marginal_out=None, zexp_out=None, tensor_cores=True,
                  use_graph=False, k_range=None):
    """Host mode (default): returns (marginal, zexp) float64 numpy arrays with
    all problems back to back.  Device mode: pass torch float64 CUDA tensors
    as ``marginal_out`` / ``zexp_out``; the call does not synchronise.
    ``k_range`` = (lo, hi): sum only the cut-index terms in [lo, hi)
    (hi = 0: to the end) -- a partial result of a split contraction."""
    lo, hi = k_range if k_range is not None else (0, 0)
    on_dev = marginal_out is not None and hasattr(marginal_out, "data_ptr")
    if on_dev:
        opts = ccs_recomb_opts(precision, 1, 0 if tensor_cores else 1, int(use_graph), lo, hi)
        ctx.check(lib().ccs_recombine(ctx.h, plan.h, res.h, C.byref(opts),
                                      C.c_void_p(marginal_out.data_ptr()),
                                      C.c_void_p(zexp_out.data_ptr() if zexp_out is not None else None)),
                  "ccs_recombine")
        return marginal_out, zexp_out
    nm = sum(1 << len(p.marginal) for p in plan.problems)
    nz = sum(len(getattr(p, "zstrings", []) or []) for p in plan.problems)
    marg = np.zeros(max(nm, 1))
    zexp = np.zeros(max(nz, 1))
    opts = ccs_recomb_opts(precision, 0, 0 if tensor_cores else 1, int(use_graph), lo, hi)
    ctx.check(lib().ccs_recombine(ctx.h, plan.h, res.h, C.byref(opts),
                                  marg.ctypes.data_as(C.c_void_p), zexp.ctypes.data_as(C.c_void_p)),
              "ccs_recombine")
    return marg[:nm], zexp[:nz]


def ccs_plan_counts(ctx, plan, problem=0):
    nf, nc = C.c_int(), C.c_int()
    ctx.check(lib().ccs_plan_counts(ctx.h, plan.h, problem, C.byref(nf), C.byref(nc)), "ccs_plan_counts")
    return nf.value, nc.value


def ccs_fragment_info_get(ctx, plan, problem, fragment):
    info = ccs_fragment_info()
    ctx.check(lib().ccs_fragment_info_get(ctx.h, plan.h, problem, fragment, C.byref(info)),
              "ccs_fragment_info_get")
    return {n: getattr(info, n) for n, _ in ccs_fragment_info._fields_}


def ccs_plan_cuts(ctx, plan, problem=0):
    buf = (ccs_cut * 64)()
    n = ctx.check(lib().ccs_plan_cuts(ctx.h, plan.h, problem, buf, 64), "ccs_plan_cuts")
    return [(buf[i].qubit, buf[i].gate_index) for i in range(n)]


def ccs_fragment_wires(ctx, plan, problem, fragment):
    n = ccs_fragment_info_get(ctx, plan, problem, fragment)["n_wires"]
    buf = np.zeros(2 * n, np.uint32)
    ctx.check(lib().ccs_fragment_wires(ctx.h, plan.h, problem, fragment,
                                       buf.ctypes.data_as(C.POINTER(C.c_uint32))), "ccs_fragment_wires")
    return [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(n)]


def ccs_get_tableau(ctx, res, problem, fragment, variant):
    n = ccs_fragment_info_get(ctx, res.plan, problem, fragment)["n_wires"]
    out = np.zeros((2 * n, 2 * n + 1), np.uint8)
    ctx.check(lib().ccs_get_tableau(ctx.h, res.h, problem, fragment, variant,
                                    out.ctypes.data_as(C.c_void_p)), "ccs_get_tableau")
    return out


def ccs_get_outcome_space(ctx, res, problem, fragment, variant):
    off = C.c_uint64()
    basis = (C.c_uint64 * 64)()
    rank = C.c_int()
    ctx.check(lib().ccs_get_outcome_space(ctx.h, res.h, problem, fragment, variant, C.byref(off),
                                          basis, C.byref(rank)), "ccs_get_outcome_space")
    return int(off.value), [int(basis[i]) for i in range(rank.value)], rank.value


def ccs_get_counts(ctx, res, problem, fragment, variant):
    nA = ccs_fragment_info_get(ctx, res.plan, problem, fragment)["n_meas"]
    out = np.zeros(1 << nA, np.uint32)
    ctx.check(lib().ccs_get_counts(ctx.h, res.h, problem, fragment, variant,
                                   out.ctypes.data_as(C.c_void_p)), "ccs_get_counts")
    return out


def ccs_get_dist(ctx, res, problem, fragment, variant):
    nA = ccs_fragment_info_get(ctx, res.plan, problem, fragment)["n_meas"]
    out = np.zeros(1 << nA, np.float32)
    ctx.check(lib().ccs_get_dist(ctx.h, res.h, problem, fragment, variant,
                                 out.ctypes.data_as(C.c_void_p)), "ccs_get_dist")
    return out


def ccs_get_zvals(ctx, res, problem, fragment, variant):
    """Z-string values of one variant: [string][subset of quantum outputs]."""
    info = ccs_fragment_info_get(ctx, res.plan, problem, fragment)
    out = np.zeros((info["n_zstrings"], 1 << info["n_qout"]), np.float32)
    ctx.check(lib().ccs_get_zvals(ctx.h, res.h, problem, fragment, variant, out.ctypes.data_as(C.c_void_p)),
              "ccs_get_zvals")
    return out


def ccs_get_tensor(ctx, res, problem, fragment):
    info = ccs_fragment_info_get(ctx, res.plan, problem, fragment)
    out = np.zeros((1 << info["n_marg"], 4 ** info["n_slots"]), np.float32)
    ctx.check(lib().ccs_get_tensor(ctx.h, res.h, problem, fragment, out.ctypes.data_as(C.c_void_p)),
              "ccs_get_tensor")
    return out


def ccs_set_profiling(ctx, on=True):
    ctx.check(lib().ccs_set_profiling(ctx.h, int(on)), "ccs_set_profiling")


def ccs_get_stage_times(ctx):
    """{stage: ms} of the last profiled calls (stages that did not run are absent)."""
    buf = (C.c_double * 8)()
    n = ctx.check(lib().ccs_get_stage_times(ctx.h, buf, 8), "ccs_get_stage_times")
    return {STAGES[i]: buf[i] for i in range(n) if buf[i] >= 0}


def ccs_cut_candidates(ctx, problem, max_cuts=12, max_nc_width=10, cap=64):
    """[(cuts, estimated cost)] from the cut search, cheapest first."""
    p, keep = _pack_problem(problem)
    opts = ccs_cut_opts(max_cuts, max_nc_width, 0)
    cuts = (ccs_cut * (cap * 16))()
    offs = (C.c_int * (cap + 1))()
    costs = (C.c_double * cap)()
    n = ctx.check(lib().ccs_cut_candidates(ctx.h, C.byref(p), C.byref(opts), cuts, cap * 16, offs, costs, cap),
                  "ccs_cut_candidates")
    return [([(cuts[j].qubit, cuts[j].gate_index) for j in range(offs[i], offs[i + 1])], costs[i])
            for i in range(n)]


def ccs_recombine_noalloc(ctx, plan, res, marginal_out, zexp_out=None, precision=CCS_FP32):
    """Recombination into caller-owned device buffers (torch float64 CUDA
    tensors) with no device allocation by the library; asynchronous."""
    ctx.check(lib().ccs_recombine_noalloc(ctx.h, plan.h, res.h, precision,
                                          C.c_void_p(marginal_out.data_ptr()),
                                          C.c_void_p(zexp_out.data_ptr() if zexp_out is not None else None)),
              "ccs_recombine_noalloc")
    return marginal_out, zexp_out


def ccs_ml_correct(ctx, plan, res, which=CCS_ML_SAMPLED):
    """Maximum-likelihood correction of the result's fragment models in place
    (Sec. V-C); asynchronous on the context stream."""
    ctx.check(lib().ccs_ml_correct(ctx.h, plan.h, res.h, which), "ccs_ml_correct")


def ccs_get_tuning(ctx, res):
    """(threads per tableau CTA, words per op per thread, shots per sampling CTA,
    threads per hub-sampler CTA (negative: byte counters), 1 if every variant
    simulates its whole circuit else 0)."""
    t, wpo, spc, hub, vp = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    ctx.check(lib().ccs_get_tuning(ctx.h, res.h, C.byref(t), C.byref(wpo), C.byref(spc), C.byref(hub),
                                   C.byref(vp)), "ccs_get_tuning")
    return t.value, wpo.value, spc.value, hub.value, vp.value


def ccs_get_operand(ctx, res, problem, fragment):
    info = ccs_fragment_info_get(ctx, res.plan, problem, fragment)
    out = np.zeros((1 << info["n_marg"], 4 ** info["n_slots"]), np.float32)
    ctx.check(lib().ccs_get_operand(ctx.h, res.h, problem, fragment, out.ctypes.data_as(C.c_void_p)),
              "ccs_get_operand")
    return out


# --- learned cut scorer --------------------------------------------------------
class ccs_graph_batch(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_graphs", C.c_int32), ("x", C.POINTER(C.c_float)),
                ("rowptr", C.POINTER(C.c_int32)), ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_float)),
                ("val_t", C.POINTER(C.c_float)), ("graph_off", C.POINTER(C.c_int32)),
                ("glob", C.POINTER(C.c_float))]


_MPNN_SIGS = {
    "ccs_mpnn_num_params": ([], C.c_int),
    "ccs_mpnn_create": ([C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p)], C.c_int),
    "ccs_mpnn_free": ([C.c_void_p], None),
    "ccs_mpnn_params": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "ccs_mpnn_set_params": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "ccs_mpnn_forward": ([C.c_void_p, C.c_void_p, C.POINTER(ccs_graph_batch), C.c_void_p], C.c_int),
    "ccs_mpnn_gradient": ([C.c_void_p, C.c_void_p, C.POINTER(ccs_graph_batch), C.c_void_p, C.c_void_p,
                           C.c_void_p], C.c_int),
    "ccs_mpnn_train_step": ([C.c_void_p, C.c_void_p, C.POINTER(ccs_graph_batch), C.c_void_p, C.c_float,
                             C.c_void_p], C.c_int),
    "ccs_featurize": ([C.c_void_p, C.POINTER(ccs_problem), C.POINTER(ccs_cut), C.c_int, C.c_void_p, C.c_void_p,
                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "ccs_set_cut_model": ([C.c_void_p, C.c_void_p], C.c_int),
}
EXPORTS += list(_MPNN_SIGS)


def _mpnn_lib():
    L = lib()
    if not getattr(L, "_mpnn_bound", False):
        for name, (args, res) in _MPNN_SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        L._mpnn_bound = True
    return L


class Graph:
    """Features of one circuit under one cut set (numpy arrays)."""

    def __init__(self, x, rowptr, col, val, val_t, glob):
        self.x, self.rowptr, self.col, self.val, self.val_t, self.glob = x, rowptr, col, val, val_t, glob


def ccs_featurize(ctx, problem, cuts):
    p, keep = _pack_problem(problem)
    n = problem.circuit.n_qubits
    cap = max(16, 2 * sum(1 for g in problem.circuit.gates if g[0] in (6, 7)))
    x = np.zeros((n, 8), np.float32)
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(cap, np.int32)
    val = np.zeros(cap, np.float32)
    val_t = np.zeros(cap, np.float32)
    glob = np.zeros(8, np.float32)
    cc = (ccs_cut * max(1, len(cuts)))(*[ccs_cut(q, g) for q, g in cuts])
    f = lambda a: a.ctypes.data_as(C.c_void_p)
    nnz = ctx.check(_mpnn_lib().ccs_featurize(ctx.h, C.byref(p), cc, len(cuts), f(x), f(rowptr), f(col), f(val),
                                              f(val_t), cap, f(glob)), "ccs_featurize")
    return Graph(x, rowptr, col[:nnz].copy(), val[:nnz].copy(), val_t[:nnz].copy(), glob)


def make_batch(graphs):
    """Concatenate graphs into block-diagonal batch arrays (kept alive on the struct)."""
    xs, rps, cols, vals, vts, gl, goff = [], [0], [], [], [], [], [0]
    for g in graphs:
        base, e0 = goff[-1], rps[-1]
        xs.append(g.x)
        rps += list(e0 + g.rowptr[1:])
        cols.append(g.col + base)
        vals.append(g.val)
        vts.append(g.val_t)
        gl.append(g.glob)
        goff.append(base + g.x.shape[0])
    arrs = dict(x=np.ascontiguousarray(np.concatenate(xs), np.float32), rowptr=np.asarray(rps, np.int32),
                col=np.ascontiguousarray(np.concatenate(cols), np.int32),
                val=np.ascontiguousarray(np.concatenate(vals), np.float32),
                val_t=np.ascontiguousarray(np.concatenate(vts), np.float32),
                graph_off=np.asarray(goff, np.int32), glob=np.ascontiguousarray(np.stack(gl), np.float32))
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    b = ccs_graph_batch(goff[-1], len(graphs), P(arrs["x"], C.c_float), P(arrs["rowptr"], C.c_int32),
                        P(arrs["col"], C.c_int32), P(arrs["val"], C.c_float), P(arrs["val_t"], C.c_float),
                        P(arrs["graph_off"], C.c_int32), P(arrs["glob"], C.c_float))
    b._arrays = arrs
    return b


class Mpnn:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def __del__(self):
        try:
            if self.h:
                _mpnn_lib().ccs_mpnn_free(self.h)
        except Exception:
            pass


def ccs_mpnn_num_params():
    return _mpnn_lib().ccs_mpnn_num_params()


def ccs_mpnn_create(ctx, seed=0):
    h = C.c_void_p()
    ctx.check(_mpnn_lib().ccs_mpnn_create(ctx.h, seed, C.byref(h)), "ccs_mpnn_create")
    return Mpnn(ctx, h)


def ccs_mpnn_params(ctx, net):
    out = np.zeros(ccs_mpnn_num_params(), np.float32)
    ctx.check(_mpnn_lib().ccs_mpnn_params(ctx.h, net.h, out.ctypes.data_as(C.c_void_p)), "ccs_mpnn_params")
    return out


def ccs_mpnn_set_params(ctx, net, params):
    p = np.ascontiguousarray(params, np.float32)
    ctx.check(_mpnn_lib().ccs_mpnn_set_params(ctx.h, net.h, p.ctypes.data_as(C.c_void_p)), "ccs_mpnn_set_params")


def ccs_mpnn_forward(ctx, net, batch):
    out = np.zeros(batch.n_graphs, np.float32)
    ctx.check(_mpnn_lib().ccs_mpnn_forward(ctx.h, net.h, C.byref(batch), out.ctypes.data_as(C.c_void_p)),
              "ccs_mpnn_forward")
    return out


def ccs_mpnn_gradient(ctx, net, batch, target):
    t = np.ascontiguousarray(target, np.float32)
    loss = np.zeros(1, np.float32)
    grad = np.zeros(ccs_mpnn_num_params(), np.float32)
    ctx.check(_mpnn_lib().ccs_mpnn_gradient(ctx.h, net.h, C.byref(batch), t.ctypes.data_as(C.c_void_p),
                                            loss.ctypes.data_as(C.c_void_p), grad.ctypes.data_as(C.c_void_p)),
              "ccs_mpnn_gradient")
    return float(loss[0]), grad


def ccs_mpnn_train_step(ctx, net, batch, target, lr=1e-3):
    t = np.ascontiguousarray(target, np.float32)
    loss = np.zeros(1, np.float32)
    ctx.check(_mpnn_lib().ccs_mpnn_train_step(ctx.h, net.h, C.byref(batch), t.ctypes.data_as(C.c_void_p), lr,
                                              loss.ctypes.data_as(C.c_void_p)), "ccs_mpnn_train_step")
    return float(loss[0])


def ccs_set_cut_model(ctx, net):
    ctx.check(_mpnn_lib().ccs_set_cut_model(ctx.h, net.h if net is not None else None), "ccs_set_cut_model")


def ccs_launch_count():
    """Kernels the library has launched in this process (graph replays count their nodes)."""
    L = lib()
    L.ccs_launch_count.restype = C.c_longlong
    L.ccs_launch_count.argtypes = []
    return int(L.ccs_launch_count())


def load_cut_scorer(ctx, path):
    """A scorer with the parameters saved by learned_cuts (npz 'params')."""
    net = ccs_mpnn_create(ctx)
    ccs_mpnn_set_params(ctx, net, np.load(path)["params"])
    return net
