"""Failure detection of the tensor-core pipelines without a GPU fault: every
barrier wait of the TMA-fed tcgen05 kernels is bounded (tn_set_wait_limit).
With the bound set to zero polls every pipeline wait gives up at once: the
kernel records an error code, drains the copies and MMAs it already issued,
releases its TMEM and exits, and the host call returns TN_ETIMEOUT.  The
context stays usable: with the default bound restored, the same call gives
the right result (against an FP64 einsum / the state-vector oracle)."""
import numpy as np
import pytest

import tn_inputs as I

from _lib import tnlib

pytestmark = pytest.mark.gpu
TN_ETIMEOUT = 5
LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def _pair_case(nm, nn, nk, seed):
    rng = np.random.default_rng(seed)
    labels = list(range(nm + nn + nk))
    M, N, K = labels[:nm], labels[nm:nm + nn], labels[nm + nn:]
    la = [int(x) for x in rng.permutation(M + K)]
    lb = [int(x) for x in rng.permutation(K + N)]
    lc = [int(x) for x in rng.permutation(M + N)]
    A = I.random_tensor(len(la), seed * 3 + 1).astype(np.complex64)
    B = I.random_tensor(len(lb), seed * 3 + 2).astype(np.complex64)
    sub = lambda ls: "".join(LETTERS[x] for x in ls)
    ref = np.einsum(f"{sub(la)},{sub(lb)}->{sub(lc)}", A.astype(np.complex128).reshape((2,) * len(la)),
                    B.astype(np.complex128).reshape((2,) * len(lb)))
    return la, lb, lc, A, B, ref.reshape(-1)


# (shape, precision): the chunked split kernel, the one-tile-per-CTA scaled
# kernel (fewer than 296 tiles) and the persistent scaled kernel (512 tiles)
CASES = [((9, 8, 9), "split_bf16"), ((9, 7, 6), "scaled_fp16"), ((16, 7, 6), "scaled_fp16")]


@pytest.mark.parametrize("shape,precision", CASES)
def test_expired_pipeline_wait_returns_etimeout_then_the_call_is_correct(shape, precision):
    import torch
    T = tnlib()
    la, lb, lc, A, B, ref = _pair_case(*shape, seed=sum(shape))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(1 << len(lc), dtype=torch.complex64, device="cuda")
    try:
        T.set_wait_limit(0)
        with pytest.raises(T.TnError) as ei:
            T.contract_pair(dA, la, dB, lb, dC, lc, precision=precision, algo="fused_tc")
        assert ei.value.status == TN_ETIMEOUT, ei.value
    finally:
        T.set_wait_limit(-1)
    torch.cuda.synchronize()
    T.contract_pair(dA, la, dB, lb, dC, lc, precision=precision, algo="fused_tc")
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= (1e-4 if precision.startswith("split") else 2e-2), err


def test_expired_wait_in_an_amplitude_call_returns_etimeout_then_the_call_is_correct():
    """The same through tn_contract_amplitudes (split bf16, 4x5 grid, depth
    1+16+1, six sliced indices, six open qubits: nine tensor-core steps)
    against the state vector."""
    T = tnlib()
    from oracle import circuit as OC
    from oracle import statevector as SV
    rows, cols, depth, seed = 4, 5, 16, 2
    n = rows * cols
    open_q = list(range(n - 6, n))
    c = T.random_circuit(rows, cols, depth, seed)
    p = T.plan(T.build_network(c, open_q), num_sliced=6, search_trials=16, seed=1)
    words = I.bitstrings(n, 2, seed)
    try:
        T.set_wait_limit(0)
        with pytest.raises(T.TnError) as ei:
            p.contract_amplitudes(words, precision="split_bf16")
        assert ei.value.status == TN_ETIMEOUT, ei.value
    finally:
        T.set_wait_limit(-1)
    got, rep = p.contract_amplitudes(words, precision="split_bf16", report=True, profile=True)
    assert rep["class_launches"][2] > 0, rep["class_launches"]  # the tensor-core class ran
    ref = SV.amplitudes(SV.simulate(OC.random_circuit(rows, cols, depth, seed), n), n,
                        [I.bits_of(w, n) for w in words], open_q)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-4, err
