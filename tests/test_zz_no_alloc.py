"""The allocation-free tensor-core contraction (tn_contract_pair_noalloc).

Some callers cannot let the library allocate device memory (a framework's
caching allocator already holding the free HBM, a serving loop with a fixed
budget, code next to a graph capture); this entry point takes its scratch
from a static device array.  Here it must agree with the allocating entry
point, call after call, and reject operands too large for the array.  The
file name sorts last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

import tn_inputs as I

from _lib import tnlib

pytestmark = pytest.mark.gpu
LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def _operands(nm, nn, nk, seed):
    rng = np.random.default_rng(seed)
    labels = list(range(nm + nn + nk))
    M, N, K = labels[:nm], labels[nm:nm + nn], labels[nm + nn:]
    la = [int(x) for x in rng.permutation(M + K)]
    lb = [int(x) for x in rng.permutation(K + N)]
    lc = [int(x) for x in rng.permutation(M + N)]
    A = I.random_tensor(len(la), seed + 1).astype(np.complex64)
    B = I.random_tensor(len(lb), seed + 2).astype(np.complex64)
    sub = lambda ls: "".join(LETTERS[x] for x in ls)
    ref = np.einsum(f"{sub(la)},{sub(lb)}->{sub(lc)}", A.astype(np.complex128).reshape((2,) * len(la)),
                    B.astype(np.complex128).reshape((2,) * len(lb))).reshape(-1)
    return la, lb, lc, A, B, ref


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    T = tnlib()
    import torch
    for call, (nm, nn, nk) in enumerate([(10, 8, 7), (9, 6, 9)]):
        la, lb, lc, A, B, ref = _operands(nm, nn, nk, seed=40 + call)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        c_alloc = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
        c_static = torch.full_like(c_alloc, float("nan"))
        T.contract_pair(dA, la, dB, lb, c_alloc, lc, precision="split_bf16", algo="fused_tc")
        T.contract_pair_noalloc(dA, la, dB, lb, c_static, lc)
        torch.cuda.synchronize()
        got = c_static.cpu().numpy().astype(np.complex128)
        base = c_alloc.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), call
        assert np.linalg.norm(got - base) <= 1e-4 * np.linalg.norm(base), call


def test_noalloc_rejects_operands_beyond_the_static_array():
    T = tnlib()
    import torch
    # M = 2^20, K = 2^6: planes need 8 * (2^20 + 2^4) * 64 bytes > 64 MiB
    a = torch.zeros(1 << 26, dtype=torch.complex64, device="cuda")
    b = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    c = torch.zeros(1 << 24, dtype=torch.complex64, device="cuda")
    la = list(range(20)) + list(range(100, 106))
    lb = list(range(100, 106)) + list(range(200, 204))
    lc = list(range(20)) + list(range(200, 204))
    with pytest.raises(T.TnError) as e:
        T.contract_pair_noalloc(a, la, b, lb, c, lc)
    assert e.value.status == 1 and "static buffer" in str(e.value)
