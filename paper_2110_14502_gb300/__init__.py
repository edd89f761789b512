"""GB300 random-circuit tensor-network library: Python binding of include/tn.h.

The compute path lives in libtn.so (CUDA kernels for sm_103a behind a C ABI);
this package only marshals arguments.  See the docstrings of
:func:`random_circuit`, :func:`build_network`, :func:`plan` and
:meth:`Plan.contract_amplitudes`.
"""
import ctypes as C

import numpy as np

from ._abi import (PAIR_ALGO, PREC, ExecOpts, Gate, NetworkInfo, PlanInfo, PlanOpts, PrecisionReport, Report, Request,
                   RequestStats, ServerOpts, TensorLayout, TnError, check, i32array, lib, require_buffer)

__all__ = ["Circuit", "Network", "Plan", "random_circuit", "circuit_from_gates", "build_network", "plan", "select_plan",
           "contract_pair", "contract_pair_noalloc", "set_wait_limit", "Server", "TnError", "PREC", "version"]


def version():
    return lib().tn_version().decode()


def _ptr(x):
    """Device or host pointer of a torch tensor / NumPy array (no copies)."""
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


class Circuit:
    def __init__(self, handle):
        self._h = handle

    def __del__(self):
        if getattr(self, "_h", None):
            lib().tn_free_circuit(self._h)
            self._h = None

    @property
    def num_qubits(self):
        n, g = C.c_int32(), C.c_int64()
        check(lib().tn_circuit_info(self._h, C.byref(n), C.byref(g)))
        return n.value

    def gates(self):
        """List of (kind, q0, q1, theta, phi, matrix complex128)."""
        n, g = C.c_int32(), C.c_int64()
        check(lib().tn_circuit_info(self._h, C.byref(n), C.byref(g)))
        arr = (Gate * max(g.value, 1))()
        check(lib().tn_circuit_gates(self._h, arr, g.value))
        out = []
        for i in range(g.value):
            t = arr[i]
            d = 4 if t.q1 >= 0 else 2
            m = np.array(t.mat[: 2 * d * d]).view(np.complex128).reshape(d, d)
            out.append((t.kind, t.q0, t.q1, t.theta, t.phi, m))
        return out


def random_circuit(rows, cols, depth, seed):
    h = C.c_void_p()
    check(lib().tn_random_circuit(rows, cols, depth, seed, C.byref(h)))
    return Circuit(h)


def circuit_from_gates(num_qubits, gates):
    """gates: iterable of (kind:str|int, qubits tuple, theta, phi, matrix or None)."""
    gates = list(gates)
    arr = (Gate * max(len(gates), 1))()
    for i, (kind, qs, theta, phi, mat) in enumerate(gates):
        t = arr[i]
        t.kind = kind if isinstance(kind, int) else {"sqrtx": 0, "sqrty": 1, "sqrtw": 2, "fsim": 3,
                                                      "mat1": 4, "mat2": 5}[kind]
        t.q0 = qs[0]
        t.q1 = qs[1] if len(qs) > 1 else -1
        t.theta, t.phi = theta, phi
        if mat is not None:
            flat = np.asarray(mat, dtype=np.complex128).reshape(-1).view(np.float64)
            for e, v in enumerate(flat):
                t.mat[e] = v
    h = C.c_void_p()
    check(lib().tn_circuit_from_gates(num_qubits, len(gates), arr, C.byref(h)))
    return Circuit(h)


class Network:
    def __init__(self, handle, circuit):
        self._h = handle
        self.circuit = circuit

    def __del__(self):
        if getattr(self, "_h", None):
            lib().tn_free_network(self._h)
            self._h = None

    def info(self):
        i = NetworkInfo()
        check(lib().tn_network_get_info(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in NetworkInfo._fields_}

    def label_wires(self):
        n = self.info()["num_labels"]
        a = np.zeros(2 * n, dtype=np.int32)
        check(lib().tn_network_label_wires(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)), n))
        return [tuple(x) for x in a.reshape(-1, 2)]


def build_network(circuit, open_qubits=(), split_diagonal=False):
    """tn_build_network_ex: the network of <x|U|0^n> with open_qubits open;
    split_diagonal (TN_NET_SPLIT_DIAGONAL) turns every swap-times-diagonal
    two-qubit gate into a wire swap plus a rank-2 bond."""
    arr, p = i32array(open_qubits)
    h = C.c_void_p()
    check(lib().tn_build_network_ex(circuit._h, p, len(arr), 1 if split_diagonal else 0, C.byref(h)))
    return Network(h, circuit)


class Plan:
    def __init__(self, handle, network):
        self._h = handle
        self.network = network

    def __del__(self):
        if getattr(self, "_h", None):
            lib().tn_free_plan(self._h)
            self._h = None

    def info(self):
        i = PlanInfo()
        check(lib().tn_plan_get_info(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in PlanInfo._fields_}

    def sliced_wires(self):
        s = self.info()["num_sliced"]
        a = np.zeros(2 * max(s, 1), dtype=np.int32)
        check(lib().tn_plan_sliced_wires(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)), s))
        return [tuple(int(v) for v in x) for x in a[: 2 * s].reshape(-1, 2)]

    def serialize(self):
        n = C.c_size_t()
        check(lib().tn_plan_serialize(self._h, None, 0, C.byref(n)))
        buf = (C.c_uint8 * n.value)()
        check(lib().tn_plan_serialize(self._h, buf, n.value, C.byref(n)))
        return bytes(buf)

    def layout(self):
        """tn_plan_layout: ([per SSA tensor dict of phase, producer, consumer,
        log2_elems, offset, store_offset, store_log2], {"leaf_store",
        "invariant", "slice_arena", "pair_arena"} sizes in complex64 elements)."""
        info = self.info()
        nt = info["num_leaves"] + info["num_steps"]
        arr = (TensorLayout * max(nt, 1))()
        sizes = (C.c_int64 * 4)()
        check(lib().tn_plan_layout(self._h, arr, nt, sizes))
        names = [f for f, _ in TensorLayout._fields_ if f != "reserved"]
        tensors = [{f: getattr(arr[i], f) for f in names} for i in range(nt)]
        return tensors, dict(zip(("leaf_store", "invariant", "slice_arena", "pair_arena"), list(sizes)))

    def tree(self, num_gates, num_qubits):
        """(leaf raw-tensor lists, SSA pairs) of the contraction tree."""
        L = self.info()["num_leaves"]
        raw = np.zeros(2 * num_gates + num_qubits + L + 1, dtype=np.int32)  # split diagonals: two factors per gate
        tree = np.zeros(2 * max(L - 1, 1), dtype=np.int32)
        check(lib().tn_plan_tree(self._h, raw.ctypes.data_as(C.POINTER(C.c_int32)), raw.size,
                                 tree.ctypes.data_as(C.POINTER(C.c_int32)), tree.size))
        leaves, cur = [], []
        for v in raw:
            if len(leaves) == L:
                break
            if v < 0:
                leaves.append(cur)
                cur = []
            else:
                cur.append(int(v))
        return leaves, [tuple(int(x) for x in p) for p in tree[: 2 * (L - 1)].reshape(-1, 2)]

    def precision_analysis(self, bitstrings, probe_slices=4, fast="scaled_bf16", accurate="split_fp16",
                           target=1e-3):
        """tn_precision_analysis: (int8 per-step precisions for
        contract_amplitudes(step_precision=...), report dict)."""
        b = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64))
        words = (self.info()["num_qubits"] + 63) // 64
        if b.ndim == 1:
            b = b.reshape(-1, 1)
        if b.ndim != 2 or b.shape[1] != words:
            raise TnError(1, f"bitstrings must have shape (nb, {words}), got {b.shape}")
        sp = np.zeros(max(self.info()["num_steps"], 1), dtype=np.int8)
        rep = PrecisionReport()
        check(lib().tn_precision_analysis(self._h, b.ctypes.data, b.shape[0], probe_slices, PREC[fast],
                                          PREC[accurate], float(target), sp.ctypes.data, C.byref(rep)))
        return sp[: self.info()["num_steps"]], {f: getattr(rep, f) for f, _ in PrecisionReport._fields_}

    def contract_amplitudes(self, bitstrings, precision="c64", slice_begin=0, slice_count=-1,
                            units_per_group=0, stream=None, out=None, overflow_policy=0, use_graph=0,
                            profile=False, report=False, test_flag_every=0, autotune=0, handover=0,
                            step_precision=None):
        """Amplitudes of each bitstring's open batch, summed over the slice range.

        bitstrings: uint64 words, shape (nb, ceil(n/64)) -- a NumPy array (host
        I/O: result returned as complex128 NumPy (nb, 2^k), written into `out`
        when given, e.g. an array over pinned memory) or a CUDA torch tensor
        (device I/O: `out` must be a CUDA float64 tensor of nb*2^k*2 entries;
        work is queued on `stream`, a torch.cuda.Stream or raw handle).
        """
        info = self.info()
        k = info["num_open"]
        o = ExecOpts()
        o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        o.slice_begin = slice_begin
        o.slice_count = slice_count
        o.units_per_group = units_per_group
        o.overflow_policy = overflow_policy
        o.use_graph = use_graph
        o.profile = 1 if profile else 0
        o.test_flag_every = test_flag_every
        o.autotune = autotune
        o.handover = handover
        if step_precision is not None:
            sp = np.ascontiguousarray(np.asarray(step_precision, dtype=np.int8))
            if sp.shape != (info["num_steps"],):
                raise TnError(1, f"step_precision needs one entry per step ({info['num_steps']}), got {sp.shape}")
            o.step_precision = sp.ctypes.data
        if stream is not None:
            o.stream = C.c_void_p(getattr(stream, "cuda_stream", stream))
        rep = Report()
        device = hasattr(bitstrings, "is_cuda") and bitstrings.is_cuda
        words = (info["num_qubits"] + 63) // 64
        if device:
            nb = bitstrings.shape[0]
            if out is None:
                raise ValueError("device I/O needs an `out` tensor")
            if bitstrings.dim() not in (1, 2) or bitstrings.numel() != nb * words:
                raise TnError(1, f"bitstrings must have shape ({nb}, {words}) or ({nb},)")
            require_buffer(bitstrings, "bitstrings", 8 * nb * words, True, ("int64", "uint64"))
            require_buffer(out, "out", 16 * (nb << k), True, ("float64", "complex128"))
            o.device_io = 1
            check(lib().tn_contract_amplitudes(self._h, _ptr(bitstrings), nb, _ptr(out), C.byref(o), C.byref(rep)))
            res = out
        else:
            b = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64))
            if b.ndim == 1:
                b = b.reshape(-1, 1)
            if b.ndim != 2 or b.shape[1] != words:
                raise TnError(1, f"bitstrings must have shape (nb, {words}), got {b.shape}")
            nb = b.shape[0]
            if out is None:
                res = np.zeros((nb, 1 << k), dtype=np.complex128)
            else:
                require_buffer(out, "out", 16 * (nb << k), False, ("complex128",))
                res = out
            check(lib().tn_contract_amplitudes(self._h, _ptr(b), nb, _ptr(res), C.byref(o), C.byref(rep)))
        if report:
            r = {}
            for f, _ in Report._fields_:
                v = getattr(rep, f)
                r[f] = list(v) if hasattr(v, "__len__") else v
            return res, r
        return res


def plan(network, num_sliced=-1, max_log2_intermediate=0, search_trials=0, seed=0, max_log2_cmac=0.0,
         bitstrings_hint=0, order_generator=0, cap_aware_rewrites=0):
    """tn_plan: contraction order, slicing and layout of `network` (options as
    the fields of tn_plan_opts in include/tn.h)."""
    o = PlanOpts()
    o.num_sliced = num_sliced
    o.max_log2_intermediate = max_log2_intermediate
    o.search_trials = search_trials
    o.seed = seed
    o.max_log2_cmac = max_log2_cmac
    o.bitstrings_hint = bitstrings_hint
    o.order_generator = order_generator
    o.cap_aware_rewrites = cap_aware_rewrites
    h = C.c_void_p()
    check(lib().tn_plan(network._h, C.byref(o), C.byref(h)))
    return Plan(h, network)


def select_plan(network, bitstrings, seeds=(1, 2, 3, 4), probe_slices=32, precision="split_bf16", **plan_kw):
    """The fastest of several plans, measured: plan the network once per seed
    (keyword arguments as for plan()), contract the first probe_slices slices
    of `bitstrings` with each plan (one untimed call to set the plan up, one
    timed by the report's device time) and keep the plan with the shortest
    time per slice.  Returns (plan, [(seed, ms per slice, plan hash), ...]).
    The planner's model ranks plans only roughly on GB300 (its kernel rates
    depend on shapes and layouts), so a few probes of real slices choose
    better than the model alone."""
    best, best_t, table = None, None, []
    for seed in seeds:
        p = plan(network, seed=seed, **plan_kw)
        ns = min(probe_slices, p.info()["num_slices"])
        p.contract_amplitudes(bitstrings, precision=precision, slice_count=ns)
        _, rep = p.contract_amplitudes(bitstrings, precision=precision, slice_count=ns, report=True)
        t = rep["device_ms"] / ns
        table.append((seed, t, p.info()["hash"]))
        if best_t is None or t < best_t:
            best, best_t = p, t
        else:
            del p  # frees its device state
    return best, table


def _require_pair_operands(A, la, B, lb, Cout, lc):
    """Each operand is a contiguous CUDA complex64 tensor of 2^rank elements
    (ranks above 30 are left to the library to reject)."""
    for x, ls, what in ((A, la, "A"), (B, lb, "B"), (Cout, lc, "C")):
        if len(ls) <= 30:
            require_buffer(x, what, 8 << len(ls), True, ("complex64",))


def contract_pair(A, a_labels, B, b_labels, Cout, c_labels, precision="c64", algo="auto", stream=None):
    """C[c_labels] = sum over shared labels of A[a_labels] * B[b_labels] on the
    GPU; A, B, C are CUDA complex64 torch tensors (contiguous)."""
    la, pa = i32array(a_labels)
    lb, pb = i32array(b_labels)
    lc, pc = i32array(c_labels)
    _require_pair_operands(A, la, B, lb, Cout, lc)
    s = C.c_void_p(getattr(stream, "cuda_stream", stream) if stream is not None else None)
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    al = PAIR_ALGO[algo] if isinstance(algo, str) else int(algo)
    check(lib().tn_contract_pair(_ptr(A), pa, len(la), _ptr(B), pb, len(lb), _ptr(Cout), pc, len(lc),
                                 prec, al, s))
    return Cout


def contract_pair_noalloc(A, a_labels, B, b_labels, Cout, c_labels, stream=None):
    """tn_contract_pair_noalloc: the tensor-core contraction (bf16 hi+lo) with
    scratch taken from the library's static device array instead of an
    allocation; for callers that cannot let the library allocate.  Calls on
    one GPU share the array, so overlapping calls race."""
    la, pa = i32array(a_labels)
    lb, pb = i32array(b_labels)
    lc, pc = i32array(c_labels)
    _require_pair_operands(A, la, B, lb, Cout, lc)
    s = C.c_void_p(getattr(stream, "cuda_stream", stream) if stream is not None else None)
    check(lib().tn_contract_pair_noalloc(_ptr(A), pa, len(la), _ptr(B), pb, len(lb), _ptr(Cout), pc, len(lc), s))
    return Cout


def set_wait_limit(polls=-1):
    """tn_set_wait_limit: bound on the polls of every pipeline wait of the TMA
    tensor-core kernels on the current GPU (-1: the default 2^24; 0: every
    such wait gives up at once and the call returns TN_ETIMEOUT)."""
    check(lib().tn_set_wait_limit(int(polls)))


class Server:
    """Continuous-batching amplitude server (tn_server_*): requests for seeded
    random circuits of any grid and depth are planned, admitted by device
    memory and in-flight slots, and interleaved slice quantum by quantum."""

    def __init__(self, max_inflight=4, slices_per_quantum=64, precision="c64", plan_trials=16,
                 hbm_budget_bytes=0, max_log2_cmac=0.0, max_log2_intermediate=0, planner_threads=0,
                 over_cap_policy=0):
        o = ServerOpts()
        o.max_inflight = max_inflight
        o.slices_per_quantum = slices_per_quantum
        o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        o.plan_trials = plan_trials
        o.hbm_budget_bytes = hbm_budget_bytes
        o.max_log2_cmac = max_log2_cmac
        o.max_log2_intermediate = max_log2_intermediate
        o.planner_threads = planner_threads
        o.over_cap_policy = over_cap_policy
        h = C.c_void_p()
        check(lib().tn_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._k = {}

    def submit(self, rows, cols, depth, seed, num_open, bitstrings, precision=None, fidelity=0.0):
        b = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64))
        if b.ndim == 1:
            b = b.reshape(-1, 1)
        words = max(1, (rows * cols + 63) // 64)
        if b.ndim != 2 or b.shape[1] != words:
            raise TnError(1, f"bitstrings must have shape (nb, {words}), got {b.shape}")
        r = Request()
        r.rows, r.cols, r.depth, r.num_open, r.seed = rows, cols, depth, num_open, seed
        r.nb = b.shape[0]
        r.bitstrings = b.ctypes.data
        r.precision = -1 if precision is None else (PREC[precision] if isinstance(precision, str) else int(precision))
        r.fidelity = float(fidelity)
        t = C.c_int64()
        check(lib().tn_submit(self._h, C.byref(r), C.byref(t)))
        self._k[t.value] = (b.shape[0], num_open)
        return t.value

    def poll(self, ticket):
        d = C.c_int32()
        check(lib().tn_poll(self._h, ticket, C.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout=0.0):
        """(complex128 amplitudes (nb, 2^num_open), stats dict); raises TnError
        with the request's status when it failed."""
        nb, k = self._k[ticket]
        out = np.zeros((nb, 1 << k), dtype=np.complex128)
        st = RequestStats()
        status = lib().tn_wait(self._h, ticket, out.ctypes.data, out.size, C.byref(st), timeout)
        if status != 5:  # TN_ETIMEOUT keeps the ticket open for a later wait
            del self._k[ticket]
        stats = {f: getattr(st, f) for f, _ in RequestStats._fields_}
        if status != 0:
            raise TnError(status, lib().tn_last_error().decode())
        return out, stats

    def close(self):
        if getattr(self, "_h", None):
            lib().tn_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
