"""ctypes declarations of the C ABI in include/tn.h (argument marshalling only).

Every computation happens in libtn.so; this module converts Python/NumPy/
torch arguments to pointers and sizes and raises on a non-zero tn_status.
Importing it fails loudly when the compiled library is missing: there is no
CPU fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtn.so")

TN_OK = 0
STATUS = {0: "TN_OK", 1: "TN_EINVAL", 2: "TN_ENOMEM", 3: "TN_EHBM", 4: "TN_ECUDA", 5: "TN_ETIMEOUT",
          6: "TN_ETOOBIG", 7: "TN_EOVERFLOW", 8: "TN_ENOTREADY", 9: "TN_ENODEVICE", 10: "TN_EINTERNAL"}
GATE_KINDS = {"sqrtx": 0, "sqrty": 1, "sqrtw": 2, "fsim": 3, "mat1": 4, "mat2": 5}
PREC = {"c64": 0, "split_bf16": 1, "split_fp16": 2, "scaled_fp16": 3, "scaled_bf16": 4}
PAIR_ALGO = {"auto": 0, "fused_simt": 1, "vector": 2, "fused_tc": 3, "unfused": 4, "gather_tc": 5, "reduce": 6}


class TnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Gate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32), ("reserved", C.c_int32),
                ("theta", C.c_double), ("phi", C.c_double), ("mat", C.c_double * 32)]


class NetworkInfo(C.Structure):
    _fields_ = [("num_qubits", C.c_int32), ("num_open", C.c_int32), ("num_leaves", C.c_int32),
                ("num_labels", C.c_int32), ("max_leaf_rank", C.c_int32), ("num_closed", C.c_int32)]


class PlanOpts(C.Structure):
    _fields_ = [("num_sliced", C.c_int32), ("max_log2_intermediate", C.c_int32), ("search_trials", C.c_int32),
                ("bitstrings_hint", C.c_int32), ("seed", C.c_uint64), ("max_log2_cmac", C.c_double),
                ("order_generator", C.c_int32), ("cap_aware_rewrites", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("num_qubits", C.c_int32), ("num_open", C.c_int32), ("num_sliced", C.c_int32),
                ("num_steps", C.c_int32), ("num_leaves", C.c_int32), ("max_log2_intermediate", C.c_int32),
                ("num_slices", C.c_int64), ("cmac_per_slice", C.c_double), ("flops_per_slice", C.c_double),
                ("log2_cmac_total", C.c_double), ("footprint_bytes_per_unit", C.c_int64), ("hash", C.c_uint64),
                ("num_dense_steps", C.c_int32), ("num_vector_steps", C.c_int32)]


class TensorLayout(C.Structure):
    _fields_ = [("phase", C.c_int32), ("producer", C.c_int32), ("consumer", C.c_int32), ("log2_elems", C.c_int32),
                ("offset", C.c_int64), ("store_offset", C.c_int64), ("store_log2", C.c_int32),
                ("step_class", C.c_int32), ("log2_m", C.c_int32), ("log2_n", C.c_int32), ("log2_k", C.c_int32),
                ("reserved", C.c_int32)]


class ExecOpts(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("precision", C.c_int32), ("device_io", C.c_int32),
                ("slice_begin", C.c_int64), ("slice_count", C.c_int64), ("units_per_group", C.c_int32),
                ("overflow_policy", C.c_int32), ("use_graph", C.c_int32), ("profile", C.c_int32),
                ("test_flag_every", C.c_int32), ("autotune", C.c_int32), ("handover", C.c_int32),
                ("reserved3", C.c_int32), ("step_precision", C.c_void_p)]


class ServerOpts(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("slices_per_quantum", C.c_int32), ("precision", C.c_int32),
                ("plan_trials", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("max_log2_cmac", C.c_double),
                ("max_log2_intermediate", C.c_int32), ("planner_threads", C.c_int32),
                ("over_cap_policy", C.c_int32), ("reserved", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("depth", C.c_int32), ("num_open", C.c_int32),
                ("seed", C.c_uint64), ("nb", C.c_int64), ("bitstrings", C.c_void_p), ("precision", C.c_int32),
                ("reserved", C.c_int32), ("fidelity", C.c_double)]


class RequestStats(C.Structure):
    _fields_ = [("submit_to_done_ms", C.c_double), ("queue_ms", C.c_double), ("device_ms", C.c_double),
                ("flops", C.c_double), ("slices", C.c_int64), ("status", C.c_int32), ("num_open", C.c_int32),
                ("nb", C.c_int64), ("plan_hash", C.c_uint64), ("planned_here", C.c_int32), ("stem_reused", C.c_int32),
                ("slice_fraction", C.c_double), ("gpu_begin_ms", C.c_double), ("gpu_end_ms", C.c_double),
                ("quanta", C.c_int64), ("batched_requests", C.c_int64)]


class PrecisionReport(C.Structure):
    _fields_ = [("err_fast", C.c_double), ("err_accurate", C.c_double), ("err_mixed", C.c_double),
                ("candidate_steps", C.c_int32), ("accurate_steps", C.c_int32),
                ("accurate_flops_fraction", C.c_double), ("accurate_slice_only_steps", C.c_int32),
                ("probe_runs", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("device_ms", C.c_double), ("flops", C.c_double), ("flops_equivalent", C.c_double),
                ("units", C.c_int64), ("kernel_launches", C.c_int64), ("flagged_units", C.c_int64),
                ("discarded_units", C.c_int64), ("class_ms", C.c_double * 4), ("class_launches", C.c_int64 * 4),
                ("class_flops", C.c_double * 4), ("class_bytes", C.c_double * 4)]


P = C.c_void_p
I32P = C.POINTER(C.c_int32)
# name -> (restype, argtypes)
SIGNATURES = {
    "tn_last_error": (C.c_char_p, []),
    "tn_version": (C.c_char_p, []),
    "tn_random_circuit": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(P)]),
    "tn_circuit_from_gates": (C.c_int, [C.c_int32, C.c_int64, C.POINTER(Gate), C.POINTER(P)]),
    "tn_circuit_info": (C.c_int, [P, I32P, C.POINTER(C.c_int64)]),
    "tn_circuit_gates": (C.c_int, [P, C.POINTER(Gate), C.c_int64]),
    "tn_free_circuit": (None, [P]),
    "tn_build_network": (C.c_int, [P, I32P, C.c_int32, C.POINTER(P)]),
    "tn_build_network_ex": (C.c_int, [P, I32P, C.c_int32, C.c_int32, C.POINTER(P)]),
    "tn_network_get_info": (C.c_int, [P, C.POINTER(NetworkInfo)]),
    "tn_network_label_wires": (C.c_int, [P, I32P, C.c_int64]),
    "tn_free_network": (None, [P]),
    "tn_plan": (C.c_int, [P, C.POINTER(PlanOpts), C.POINTER(P)]),
    "tn_plan_get_info": (C.c_int, [P, C.POINTER(PlanInfo)]),
    "tn_plan_sliced_wires": (C.c_int, [P, I32P, C.c_int64]),
    "tn_plan_serialize": (C.c_int, [P, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "tn_plan_tree": (C.c_int, [P, I32P, C.c_int64, I32P, C.c_int64]),
    "tn_plan_layout": (C.c_int, [P, C.POINTER(TensorLayout), C.c_int64, C.POINTER(C.c_int64)]),
    "tn_free_plan": (None, [P]),
    "tn_contract_amplitudes": (C.c_int, [P, C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(ExecOpts),
                                         C.POINTER(Report)]),
    "tn_contract_pair": (C.c_int, [C.c_void_p, I32P, C.c_int32, C.c_void_p, I32P, C.c_int32,
                                   C.c_void_p, I32P, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "tn_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(P)]),
    "tn_submit": (C.c_int, [P, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "tn_poll": (C.c_int, [P, C.c_int64, C.POINTER(C.c_int32)]),
    "tn_wait": (C.c_int, [P, C.c_int64, C.c_void_p, C.c_int64, C.POINTER(RequestStats), C.c_double]),
    "tn_server_destroy": (None, [P]),
    "tn_contract_pair_noalloc": (C.c_int, [C.c_void_p, I32P, C.c_int32, C.c_void_p, I32P, C.c_int32,
                                           C.c_void_p, I32P, C.c_int32, C.c_void_p]),
    "tn_set_wait_limit": (C.c_int, [C.c_int64]),
    "tn_precision_analysis": (C.c_int, [P, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                        C.c_void_p, C.POINTER(PrecisionReport)]),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2110_14502_gb300.build.build()")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def check(status):
    if status != TN_OK:
        raise TnError(status, lib().tn_last_error().decode())


def require_buffer(x, what, nbytes, device, dtypes):
    """Checks a buffer before its raw pointer crosses the C ABI, which cannot
    see sizes: `x` must be a contiguous CUDA torch tensor (device=True) or a
    C-contiguous NumPy array (device=False) of one of the dtype names in
    `dtypes`, holding at least `nbytes` bytes.  Raises TnError(TN_EINVAL)."""
    if hasattr(x, "data_ptr"):
        on_dev, ok = bool(x.is_cuda), x.is_contiguous()
        dt, size = str(x.dtype).replace("torch.", ""), x.numel() * x.element_size()
    else:
        on_dev, ok = False, bool(x.flags.c_contiguous)
        dt, size = str(x.dtype), x.nbytes
    side = "a CUDA tensor" if device else "a host array"
    if on_dev != device or not ok or dt not in dtypes or size < nbytes:
        raise TnError(1, f"{what} must be {side}, contiguous, of dtype {'/'.join(dtypes)} and at least {nbytes} "
                         f"bytes (got {'device' if on_dev else 'host'}, contiguous={ok}, {dt}, {size} bytes)")


def i32array(xs):
    a = np.ascontiguousarray(np.asarray(list(xs), dtype=np.int32))
    return a, (a.ctypes.data_as(I32P) if a.size else None)
