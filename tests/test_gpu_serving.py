"""Serving (continuous batching): requests for circuits of different grids and
depths are admitted by memory and slots and interleaved slice quantum by
quantum on separate streams; a request's amplitudes must be the same alone and
in the mix, over-cap requests must fail loudly."""
import numpy as np
import pytest

import tn_inputs as I
from oracle import circuit as OC
from oracle import statevector as SV

from _lib import tnlib

pytestmark = pytest.mark.gpu


def _req(rows, cols, depth, seed, k, nb):
    n = rows * cols
    return dict(rows=rows, cols=cols, depth=depth, seed=seed, num_open=k, bitstrings=I.bitstrings(n, nb, seed))


@pytest.mark.parametrize("mode,tol", [("c64", 1e-5), ("split_bf16", 1e-4), ("scaled_fp16", 2e-2)])
def test_alone_equals_in_the_mix(mode, tol):
    T = tnlib()
    target = _req(4, 5, 12, 21, 3, 2)
    srv = T.Server(max_inflight=4, slices_per_quantum=4, precision=mode, plan_trials=8, max_log2_intermediate=12)
    try:
        alone, st = srv.wait(srv.submit(**target))
        assert st["status"] == 0 and st["slices"] >= 2
        others = [_req(4, 4, 10, 30 + i, i % 4, 1 + i % 3) for i in range(6)] + \
                 [_req(5, 4, 14, 40 + i, 2, 2) for i in range(3)]
        tickets = [srv.submit(**r) for r in others[:4]]
        tt = srv.submit(**target)
        tickets += [srv.submit(**r) for r in others[4:]]
        mixed, st2 = srv.wait(tt)
        for t in tickets:
            srv.wait(t)
    finally:
        srv.close()
    assert np.array_equal(alone, mixed)
    gates = OC.random_circuit(4, 5, 12, 21)
    n = 20
    open_q = tuple(range(n - 3, n))
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in target["bitstrings"]], open_q)
    assert np.linalg.norm(alone - ref) <= tol * np.linalg.norm(ref)


def test_over_cap_and_over_budget_requests_fail_loudly():
    T = tnlib()
    srv = T.Server(max_inflight=2, precision="c64", plan_trials=4, max_log2_cmac=20.0)
    try:
        with pytest.raises(T.TnError) as e:
            srv.wait(srv.submit(**_req(6, 6, 16, 2, 0, 1)))
        assert e.value.status == 6          # TN_ETOOBIG
        ok, st = srv.wait(srv.submit(**_req(3, 3, 4, 1, 1, 1)))
        assert st["status"] == 0
    finally:
        srv.close()
    srv = T.Server(max_inflight=2, precision="c64", plan_trials=4, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(T.TnError) as e:
            srv.wait(srv.submit(**_req(4, 4, 8, 1, 0, 1)))
        assert e.value.status == 3          # TN_EHBM
    finally:
        srv.close()


def test_stems_stay_resident_for_later_requests_of_a_circuit():
    """The second and later requests for a circuit reuse its resident stem
    (leaf tensors and phase-0 intermediates) instead of rebuilding it, also
    when they arrive together (and share a contraction); their amplitudes are
    bit-identical to those of a server that builds the stem afresh, and match
    the state vector."""
    T = tnlib()
    rows, cols, depth, seed, k = 4, 5, 12, 23, 3
    n = rows * cols
    reqs = [dict(rows=rows, cols=cols, depth=depth, seed=seed, num_open=k,
                 bitstrings=I.bitstrings(n, 2, 100 + i)) for i in range(5)]
    kw = dict(max_inflight=4, slices_per_quantum=2, precision="c64", plan_trials=8, max_log2_intermediate=12)
    srv = T.Server(**kw)
    try:
        first, st0 = srv.wait(srv.submit(**reqs[0]))
        assert st0["stem_reused"] == 0
        tickets = [srv.submit(**r) for r in reqs[1:]]
        shared = []
        for t in tickets:
            o, st = srv.wait(t)
            assert st["stem_reused"] == 1 and st["planned_here"] == 0
            shared.append(o)
    finally:
        srv.close()
    fresh = []
    for r in reqs[1:]:
        srv = T.Server(**kw)
        try:
            o, st = srv.wait(srv.submit(**r))
            assert st["stem_reused"] == 0
            fresh.append(o)
        finally:
            srv.close()
    for a, b in zip(shared, fresh):
        assert np.array_equal(a, b)
    gates = OC.random_circuit(rows, cols, depth, seed)
    psi = SV.simulate(gates, n)
    open_q = tuple(range(n - k, n))
    for r, o in zip(reqs, [first] + shared):
        ref = SV.amplitudes(psi, n, [I.bits_of(w, n) for w in r["bitstrings"]], open_q)
        assert np.linalg.norm(o - ref) <= 1e-5 * np.linalg.norm(ref)


def test_partial_fidelity_requests_serve_a_fraction_of_the_slices():
    """Fidelity by fraction: a request with fidelity f is served from the first
    ceil(f 2^S) slices.  Its amplitudes are the exact partial sum over those
    slices (the plain path on the same slice range), and over the whole
    output space their fidelity with the state vector, and the XEB of exact
    samples scored with them, are close to the served fraction."""
    T = tnlib()
    rows, cols, depth, seed = 4, 5, 14, 21
    n = rows * cols
    k = 12
    # 256 bitstrings whose closed qubits 0..7 take every value: all 2^20 amplitudes
    words = np.array([[x] for x in range(256)], dtype=np.uint64)
    kw = dict(max_inflight=2, slices_per_quantum=4, precision="c64", plan_trials=8, max_log2_intermediate=15)
    srv = T.Server(**kw)
    try:
        full, st1 = srv.wait(srv.submit(rows=rows, cols=cols, depth=depth, seed=seed, num_open=k, bitstrings=words))
        part, st = srv.wait(srv.submit(rows=rows, cols=cols, depth=depth, seed=seed, num_open=k, bitstrings=words,
                                       fidelity=0.25))
    finally:
        srv.close()
    S_all = st1["slices"]
    assert S_all >= 16 and st1["slice_fraction"] == 1.0
    m = int(np.ceil(0.25 * S_all))
    assert st["slices"] == m and abs(st["slice_fraction"] - m / S_all) < 1e-12
    # the same plan through the plain path, first m slices
    c = T.random_circuit(rows, cols, depth, seed)
    p = T.plan(T.build_network(c, list(range(n - k, n))), max_log2_intermediate=15, search_trials=8, seed=1,
               max_log2_cmac=48.0)
    assert p.info()["hash"] == st["plan_hash"]
    ref = p.contract_amplitudes(words, slice_count=m)
    assert np.linalg.norm(part - ref) <= 1e-6 * np.linalg.norm(ref)
    # amplitude of basis index x: bitstring x & 255, open index x >> 8
    a_f = part.T.reshape(-1)
    a = full.T.reshape(-1)
    gates = OC.random_circuit(rows, cols, depth, seed)
    psi = SV.simulate(gates, n)
    assert np.linalg.norm(a - psi) <= 1e-5 * np.linalg.norm(psi)
    fid = abs(np.vdot(a_f, psi)) ** 2 / (np.vdot(a_f, a_f).real * np.vdot(psi, psi).real)
    p_true = np.abs(psi) ** 2
    p_f = np.abs(a_f) ** 2 / np.sum(np.abs(a_f) ** 2)
    xeb = (2.0 ** n) * np.sum(p_true * p_f) - 1.0
    frac = m / S_all
    assert abs(fid - frac) <= 0.05 and abs(xeb - frac) <= 0.05, (fid, xeb, frac)


def test_partial_fidelity_requests_are_charged_for_the_slices_served():
    """The server's cost cap bounds the work a request is served.  The 4x5
    depth-12 circuit below plans to 2^26.38 CMAC in 2^8 slices: at full
    fidelity and at f = 0.75 it is over a 2^25.3 cap, at f = 0.25 its 64
    slices cost 2^24.38 and it is served, with the plain path's partial sum
    over the same slices."""
    import math
    T = tnlib()
    req = _req(4, 5, 12, 21, 3, 2)
    cap = 25.3
    srv = T.Server(max_inflight=2, precision="c64", plan_trials=8, max_log2_intermediate=12, max_log2_cmac=cap)
    try:
        for f in (0.0, 0.75):
            with pytest.raises(T.TnError) as e:
                srv.wait(srv.submit(**req, fidelity=f))
            assert e.value.status == 6          # TN_ETOOBIG
        part, st = srv.wait(srv.submit(**req, fidelity=0.25))
    finally:
        srv.close()
    assert st["status"] == 0 and st["slices"] == 64 and st["slice_fraction"] == 0.25
    c = T.random_circuit(4, 5, 12, 21)
    p = T.plan(T.build_network(c, [17, 18, 19]), max_log2_intermediate=12, search_trials=8, seed=1,
               max_log2_cmac=cap + 2.0)
    assert p.info()["hash"] == st["plan_hash"]
    assert math.log2(64 * p.info()["cmac_per_slice"]) <= cap
    ref = p.contract_amplitudes(req["bitstrings"], slice_count=64)
    assert np.linalg.norm(part - ref) <= 1e-6 * np.linalg.norm(ref)


def test_admitted_requests_overlap_on_the_device():
    """Continuous batching, not a queue: two admitted requests advance one
    slice quantum per scheduler turn each on their own streams, so their
    device intervals (CUDA events around the first and the last quantum)
    overlap; each result is bit-identical to the same request served alone
    and agrees with the state vector."""
    T = tnlib()
    reqs = [_req(4, 5, 14, 60 + i, 4, 2) for i in range(2)]
    srv = T.Server(max_inflight=4, slices_per_quantum=4, precision="c64", plan_trials=8, max_log2_intermediate=15)
    try:
        alone = [srv.wait(srv.submit(**r)) for r in reqs]  # also fills the plan cache
        tickets = [srv.submit(**r) for r in reqs]
        mixed = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    (o0, s0), (o1, s1) = mixed
    assert s0["quanta"] >= 8 and s1["quanta"] >= 8, (s0["quanta"], s1["quanta"])
    assert s0["gpu_end_ms"] > s0["gpu_begin_ms"] > 0 and s1["gpu_end_ms"] > s1["gpu_begin_ms"] > 0
    overlap = min(s0["gpu_end_ms"], s1["gpu_end_ms"]) - max(s0["gpu_begin_ms"], s1["gpu_begin_ms"])
    shorter = min(s0["gpu_end_ms"] - s0["gpu_begin_ms"], s1["gpu_end_ms"] - s1["gpu_begin_ms"])
    assert overlap >= 0.5 * shorter, (s0, s1)
    n = 20
    for r, (a, _), (m, _) in zip(reqs, alone, mixed):
        assert np.array_equal(a, m)
        gates = OC.random_circuit(r["rows"], r["cols"], r["depth"], r["seed"])
        ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in r["bitstrings"]],
                            tuple(range(n - 4, n)))
        assert np.linalg.norm(m - ref) <= 1e-5 * np.linalg.norm(ref)


def test_same_plan_different_circuits_keep_their_own_stems():
    """Two circuits of the same grid and depth drawn with different seeds plan
    to the same tree (the same plan hash) but have different gate matrices:
    the resident stem of one must never serve the other."""
    T = tnlib()
    reqs = [_req(4, 5, 14, 60 + i, 4, 2) for i in range(2)]
    srv = T.Server(max_inflight=2, slices_per_quantum=16, precision="c64", plan_trials=8, max_log2_intermediate=15)
    try:
        res = [srv.wait(srv.submit(**r)) for r in reqs]
        again = srv.wait(srv.submit(**reqs[0]))
    finally:
        srv.close()
    assert res[0][1]["plan_hash"] == res[1][1]["plan_hash"]
    assert res[1][1]["stem_reused"] == 0 and again[1]["stem_reused"] == 1
    assert np.array_equal(again[0], res[0][0])
    n = 20
    for r, (out, _) in zip(reqs, res):
        gates = OC.random_circuit(r["rows"], r["cols"], r["depth"], r["seed"])
        ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in r["bitstrings"]],
                            tuple(range(n - 4, n)))
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)


def test_over_cap_requests_are_served_at_partial_fidelity_when_asked():
    """over_cap_policy 1: a request whose full plan costs more than the cap is
    served from the largest leading range of slices that fits it (fidelity
    about the served fraction) instead of failing; its amplitudes are the
    plain path's partial sum over the same slices."""
    import math
    T = tnlib()
    req = _req(4, 5, 12, 21, 3, 2)
    cap = 25.3
    srv = T.Server(max_inflight=2, precision="c64", plan_trials=8, max_log2_intermediate=12, max_log2_cmac=cap,
                   over_cap_policy=1)
    try:
        part, st = srv.wait(srv.submit(**req))
    finally:
        srv.close()
    c = T.random_circuit(4, 5, 12, 21)
    p = T.plan(T.build_network(c, [17, 18, 19]), max_log2_intermediate=12, search_trials=8, seed=1,
               max_log2_cmac=1000.0)
    info = p.info()
    assert info["hash"] == st["plan_hash"]
    ns = int(math.floor(2 ** cap / info["cmac_per_slice"]))
    assert 1 <= ns < info["num_slices"] and st["slices"] == ns and st["status"] == 0
    assert abs(st["slice_fraction"] - ns / info["num_slices"]) < 1e-12
    assert math.log2(ns * info["cmac_per_slice"]) <= cap
    ref = p.contract_amplitudes(req["bitstrings"], slice_count=ns)
    assert np.linalg.norm(part - ref) <= 1e-6 * np.linalg.norm(ref)


def test_requests_for_one_circuit_share_a_contraction():
    """Requests for the same circuit, open qubits and precision that wait for
    admission together are served by one contraction (their bitstrings are
    units of the same launches): each gets exactly what it gets alone, and
    its statistics say how many requests shared the contraction."""
    T = tnlib()
    blocker = _req(4, 5, 12, 77, 2, 1)  # 256 one-slice quanta in front of the others
    target = [_req(4, 5, 12, 21, 3, 1 + i % 2) for i in range(4)]
    for i, r in enumerate(target):  # same circuit, different bitstrings
        r["bitstrings"] = I.bitstrings(20, r["bitstrings"].shape[0], 500 + i)
    srv = T.Server(max_inflight=1, slices_per_quantum=1, precision="split_bf16", plan_trials=8,
                   max_log2_intermediate=12)
    try:
        tb = srv.submit(**blocker)
        tickets = [srv.submit(**r) for r in target]
        together = [srv.wait(t) for t in tickets]
        srv.wait(tb)
        alone = [srv.wait(srv.submit(**r)) for r in target]
    finally:
        srv.close()
    assert max(st["batched_requests"] for _, st in together) >= 2, [st["batched_requests"] for _, st in together]
    assert all(st["batched_requests"] == 1 for _, st in alone)
    n = 20
    gates = OC.random_circuit(4, 5, 12, 21)
    psi = SV.simulate(gates, n)
    for r, (o, st), (a, _) in zip(target, together, alone):
        assert st["status"] == 0 and st["nb"] == r["bitstrings"].shape[0]
        assert np.array_equal(o, a)
        ref = SV.amplitudes(psi, n, [I.bits_of(w, n) for w in r["bitstrings"]], (17, 18, 19))
        assert np.linalg.norm(o - ref) <= 1e-4 * np.linalg.norm(ref)


def test_a_stem_that_does_not_fit_evicts_the_cached_ones(monkeypatch):
    """A new circuit's stem whose device allocation fails (host-side fault
    injection: TN_FAULT_ALLOC=1 fails the next allocation) evicts the cached
    stems that no request holds and is allocated once more: the request is
    served correctly, and the evicted circuit's stem is rebuilt when it
    comes back."""
    T = tnlib()
    first, second = _req(4, 5, 14, 71, 4, 2), _req(4, 5, 14, 72, 4, 2)
    srv = T.Server(max_inflight=1, slices_per_quantum=16, precision="c64", plan_trials=8, max_log2_intermediate=15)
    try:
        a, sa = srv.wait(srv.submit(**first))
        monkeypatch.setenv("TN_FAULT_ALLOC", "1")
        b, sb = srv.wait(srv.submit(**second))
        monkeypatch.delenv("TN_FAULT_ALLOC")
        a2, sa2 = srv.wait(srv.submit(**first))
    finally:
        srv.close()
    assert sa["status"] == 0 and sb["status"] == 0 and sa2["status"] == 0
    assert sa2["stem_reused"] == 0  # evicted to make room for the second circuit's stem
    assert np.array_equal(a2, a)
    n = 20
    for r, out in ((first, a), (second, b)):
        gates = OC.random_circuit(r["rows"], r["cols"], r["depth"], r["seed"])
        ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in r["bitstrings"]],
                            tuple(range(n - 4, n)))
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
