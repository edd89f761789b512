"""Parity in the benchmark's own launch configuration at full size (kept in a
file of its own that runs after the other amplitude tests)."""
import numpy as np
import pytest

import tn_inputs as I
from oracle import circuit as OC

from _lib import tnlib
from _replay import replay

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _setup(T, rows, cols, depth, cseed, open_q=(), **kw):
    c = T.random_circuit(rows, cols, depth, cseed)
    net = T.build_network(c, list(open_q))
    return T.plan(net, **kw)


def test_full_size_6x6_in_the_bench_launch_configuration():
    """The benchmark's own call -- all 1024 slices of the 6x6 plan for the
    four bitstrings, split bf16, device I/O, the default slice groups -- with
    a sampled slice recovered from it: the FP64 sum runs in slice order and a
    slice's values do not depend on the group it runs in, so the full sum
    minus the sum over every other slice is that slice up to FP64 rounding.
    Each recovered slice against the oracle's FP64 contraction."""
    import torch
    T = tnlib()
    rows, cols, depth, seed = 6, 6, 16, 2
    n = 36
    open_q = tuple(range(30, 36))
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=10, search_trials=64, seed=1)
    wires = p.sliced_wires()
    words = I.bitstrings(n, 4, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    dw = torch.from_numpy(words.astype(np.int64)).cuda()
    s_ = torch.cuda.Stream()

    def device_call(**kw):
        out = torch.empty(4 * 64 * 2, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s_):
            p.contract_amplitudes(dw, out=out, stream=s_, precision="split_bf16", **kw)
        torch.cuda.synchronize()
        return out.cpu().numpy().view(np.complex128).reshape(4, 64)

    full = device_call()
    for s, others in ((1023, [dict(slice_begin=0, slice_count=1023)]),
                      (0, [dict(slice_begin=1, slice_count=1023)])):
        rest = sum(device_call(**kw) for kw in others)
        one = full - rest
        fixed = {wires[j]: (s >> j) & 1 for j in range(len(wires))}
        for b in ((0, 3) if s else (0,)):
            ref = replay(p, gates, n, I.bits_of(words[b], n), open_q, fixed)
            assert rel(one[b], ref) <= 1e-4, (s, b, rel(one[b], ref))
