"""Pairwise fused permute-GEMM kernels against an FP64 einsum of the same
complex64 inputs (paper: Sec. "Tensor Contraction Using Fused Permutation and
Multiplication")."""
import numpy as np
import pytest

import tn_inputs as I

from _lib import tnlib

pytestmark = pytest.mark.gpu
LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def _case(nm, nn, nk, seed):
    rng = np.random.default_rng(seed)
    labels = list(range(nm + nn + nk))
    M, N, K = labels[:nm], labels[nm:nm + nn], labels[nm + nn:]
    la = list(rng.permutation(M + K))
    lb = list(rng.permutation(K + N))
    lc = list(rng.permutation(M + N))
    A = I.random_tensor(len(la), seed * 3 + 1).astype(np.complex64)
    B = I.random_tensor(len(lb), seed * 3 + 2).astype(np.complex64)
    sub = lambda ls: "".join(LETTERS[x] for x in ls)
    ref = np.einsum(f"{sub(la)},{sub(lb)}->{sub(lc)}",
                    A.astype(np.complex128).reshape((2,) * len(la)) if la else A.astype(np.complex128)[0],
                    B.astype(np.complex128).reshape((2,) * len(lb)) if lb else B.astype(np.complex128)[0])
    return la, lb, lc, A, B, np.asarray(ref).reshape(-1)


def _run(T, la, lb, lc, A, B, algo):
    import torch
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
    T.contract_pair(dA, la, dB, lb, dC, lc, precision="c64", algo=algo)
    torch.cuda.synchronize()
    return dC.cpu().numpy().astype(np.complex128)


SHAPES = [(0, 0, 0), (3, 0, 2), (0, 3, 2), (5, 5, 0), (6, 2, 2), (9, 4, 4), (7, 6, 5), (3, 7, 6), (10, 9, 3),
          (12, 8, 8), (16, 6, 7), (2, 2, 12)]


@pytest.mark.parametrize("nm,nn,nk", SHAPES)
@pytest.mark.parametrize("algo", ["auto", "fused_simt", "unfused"])
def test_pair_c64_matches_fp64(nm, nn, nk, algo):
    T = tnlib()
    la, lb, lc, A, B, ref = _case(nm, nn, nk, seed=nm * 100 + nn * 10 + nk)
    got = _run(T, la, lb, lc, A, B, algo)
    err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
    assert err <= 1e-5, err


@pytest.mark.parametrize("nm,nn,nk", [(0, 0, 0), (5, 1, 3), (12, 4, 4), (18, 2, 2), (20, 4, 2),
                                      (3, 3, 5), (11, 3, 5), (13, 2, 6), (9, 0, 7), (16, 3, 7), (10, 1, 6),
                                      (13, 5, 2), (10, 8, 1), (9, 6, 2), (3, 8, 2), (12, 7, 0), (11, 5, 1),
                                      (13, 5, 3), (6, 5, 3)])
def test_vector_kernel_matches_fp64(nm, nn, nk):
    """Streaming kernel: N, K <= 16 with the row's K values in registers,
    N <= 8 with K up to 128 consumed into running sums, N up to 256 with
    K <= 4, and N = 32 with K = 8; ragged M below one CTA's 1024 rows included."""
    T = tnlib()
    la, lb, lc, A, B, ref = _case(nm, nn, nk, seed=7 + nm + nk)
    for algo in ("vector", "auto"):
        got = _run(T, la, lb, lc, A, B, algo)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), algo


@pytest.mark.parametrize("nm,nn,nk", [(5, 3, 5), (9, 4, 3), (11, 3, 5), (12, 4, 4), (13, 2, 6), (10, 1, 6),
                                      (16, 3, 7), (18, 3, 5), (7, 0, 7), (6, 4, 3), (14, 0, 3), (15, 5, 3)])
def test_vector_kernel_contiguous_rows(nm, nn, nk):
    """Planner-style layouts (the contracted indices innermost, in one order
    in both operands): the rows of A are contiguous K runs, which the
    streaming kernel stages through shared memory; M from one 32-row group to
    several 1024-row CTAs, free index orders random."""
    T = tnlib()
    rng = np.random.default_rng(300 + 10 * nm + nk)
    labels = list(range(nm + nn + nk))
    M, N, K = labels[:nm], labels[nm:nm + nn], labels[nm + nn:]
    kk = [int(x) for x in rng.permutation(K)]
    la = [int(x) for x in rng.permutation(M)] + kk
    lb = [int(x) for x in rng.permutation(N)] + kk
    lc = [int(x) for x in rng.permutation(M + N)]
    A = I.random_tensor(len(la), 61 + nm).astype(np.complex64)
    B = I.random_tensor(len(lb), 62 + nk).astype(np.complex64)
    sub = lambda ls: "".join(LETTERS[x] for x in ls)
    ref = np.einsum(f"{sub(la)},{sub(lb)}->{sub(lc)}", A.astype(np.complex128).reshape((2,) * len(la)),
                    B.astype(np.complex128).reshape((2,) * len(lb))).reshape(-1)
    for algo in ("vector", "auto"):
        got = _run(T, la, lb, lc, A, B, algo)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), algo


@pytest.mark.parametrize("nm,nn,nk", [(0, 0, 8), (4, 2, 12), (2, 4, 9), (6, 0, 10), (0, 6, 8), (3, 3, 14),
                                      (1, 2, 16)])
def test_reduction_kernel_matches_fp64(nm, nn, nk):
    """Few outputs (M N <= 64) and a long contracted index: K spread over the
    threads of a CTA and combined with warp shuffles; random index orders."""
    T = tnlib()
    la, lb, lc, A, B, ref = _case(nm, nn, nk, seed=200 + 10 * nm + nk)
    for algo in ("reduce", "auto"):
        got = _run(T, la, lb, lc, A, B, algo)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), algo


@pytest.mark.parametrize("order", ["identity", "reversed", "interleaved"])
@pytest.mark.parametrize("algo,precision,tol", [("fused_simt", "c64", 1e-5), ("fused_tc", "split_bf16", 1e-4),
                                                ("vector", "c64", 1e-5)])
def test_permutation_corner_cases(order, algo, precision, tol):
    """Operand and output orders: identity (contracted indices innermost, free
    indices in order), fully reversed, and contracted indices interleaved with
    free ones."""
    T = tnlib()
    import torch
    nm, nn, nk = (9, 4, 3) if algo == "vector" else (9, 6, 5)
    M, N, K = list(range(nm)), list(range(nm, nm + nn)), list(range(nm + nn, nm + nn + nk))
    if order == "identity":
        la, lb, lc = M + K, N + K, M + N
    elif order == "reversed":
        la, lb, lc = (K + M)[::-1], (K + N)[::-1], (N + M)[::-1]
    else:
        la = [x for pair in zip(M, K) for x in pair] + M[len(K):]
        lb = [x for pair in zip(K, N) for x in pair] + N[len(K):] + K[len(N):]
        lc = [x for pair in zip(N, M) for x in pair] + M[len(N):]
    A = I.random_tensor(len(la), 41).astype(np.complex64)
    B = I.random_tensor(len(lb), 42).astype(np.complex64)
    sub = lambda ls: "".join(LETTERS[x] for x in ls)
    ref = np.einsum(f"{sub(la)},{sub(lb)}->{sub(lc)}", A.astype(np.complex128).reshape((2,) * len(la)),
                    B.astype(np.complex128).reshape((2,) * len(lb))).reshape(-1)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
    T.contract_pair(dA, la, dB, lb, dC, lc, precision=precision, algo=algo)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), order


def test_pair_rejects_bad_labels():
    T = tnlib()
    import torch
    a = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TnError):
        T.contract_pair(a, [0, 1], a, [1, 2], a, [0, 1], algo="auto")   # shared label in C
    with pytest.raises(T.TnError):
        T.contract_pair(a, [0, 0], a, [1, 2], a, [1, 2], algo="auto")   # repeated label


TC_SHAPES = [(7, 4, 3), (7, 6, 5), (8, 7, 6), (10, 6, 9), (9, 9, 4), (12, 8, 10), (14, 7, 7), (7, 5, 4), (8, 8, 12),
             (15, 8, 6), (16, 7, 5), (13, 9, 8),  # >= 296 tiles: persistent CTAs
             (7, 4, 14), (7, 5, 16),              # long K: chunked accumulation keeps the error flat
             (12, 5, 3), (16, 7, 3), (10, 6, 3)]  # K = 8: operand rows by bulk copies, zero upper K half


@pytest.mark.parametrize("nm,nn,nk", TC_SHAPES)
@pytest.mark.parametrize("algo", ["fused_tc", "gather_tc"])
def test_tcgen05_split_bf16_matches_fp64(nm, nn, nk, algo):
    """tcgen05 kernel, bf16 hi+lo split products with FP32 accumulation:
    relative L2 error <= 1e-4 (the split-precision bound)."""
    T = tnlib()
    import torch
    la, lb, lc, A, B, ref = _case(nm, nn, nk, seed=1000 + nm * 100 + nn * 10 + nk)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
    T.contract_pair(dA, la, dB, lb, dC, lc, precision="split_bf16", algo=algo)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-4, err



@pytest.mark.parametrize("nk", [10, 14, 16])
def test_split_error_does_not_grow_with_k(nk):
    """The tensor core's FP32 accumulation truncates, so a long K chain drifts
    toward zero; the split-precision kernel accumulates chunks in TMEM and folds
    them with round-to-nearest adds.  The error must stay at the split level
    (a few 1e-6) and carry no systematic shrink of |C|."""
    T = tnlib()
    import torch
    la, lb, lc, A, B, ref = _case(7, 5, nk, seed=77 + nk)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
    T.contract_pair(dA, la, dB, lb, dC, lc, precision="split_bf16", algo="fused_tc")
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5
    bias = float(np.mean((np.abs(got) - np.abs(ref)) / np.abs(ref)))
    assert abs(bias) <= 1e-5


PAIR_BOUND = {"split_fp16": 2e-5, "scaled_fp16": 2e-3, "scaled_bf16": 1.5e-2}


@pytest.mark.parametrize("mode", list(PAIR_BOUND))
@pytest.mark.parametrize("nm,nn,nk", [(7, 4, 3), (8, 7, 6), (9, 5, 11), (13, 9, 8), (14, 5, 3)])
def test_tensor_core_precisions_vs_fp64(mode, nm, nn, nk):
    """The TMA tensor-core kernel in the precisions that scale operands by
    their exact maxima: split fp16 (four planes, chunked accumulation) and one
    16-bit product per real product (two planes, double-buffered persistent
    CTAs for the last shape), against FP64 einsum.  Operands are scaled by
    2^-40 so that unscaled fp16 would underflow."""
    T = tnlib()
    import torch
    la, lb, lc, A, B, ref = _case(nm, nn, nk, seed=5 * nm + nk)
    s = np.float32(2.0 ** -40)
    dA = torch.from_numpy(A * s).cuda()
    dB = torch.from_numpy(B * s).cuda()
    dC = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
    T.contract_pair(dA, la, dB, lb, dC, lc, precision=mode, algo="fused_tc")
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.complex128) / (float(s) ** 2)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= PAIR_BOUND[mode], mode


def test_rank_30_operand_sampled_outputs():
    """Largest operand rank (30: 2^30 complex64 = 8 GiB) through the
    tensor-core and FP32 kernels: M = 2^20, N = 2^6, K = 2^10 with random
    index orders; 64 sampled outputs against FP64 dot products of the same
    input values on the host."""
    T = tnlib()
    import torch
    nm, nn, nk = 20, 6, 10
    rng = np.random.default_rng(30)
    labels = list(range(nm + nn + nk))
    M, N, K = labels[:nm], labels[nm:nm + nn], labels[nm + nn:]
    la = [int(x) for x in rng.permutation(M + K)]
    lb = [int(x) for x in rng.permutation(K + N)]
    lc = [int(x) for x in rng.permutation(M + N)]
    g = torch.Generator(device="cuda").manual_seed(30)
    dA = torch.randn(1 << len(la), dtype=torch.complex64, device="cuda", generator=g)
    dB = torch.randn(1 << len(lb), dtype=torch.complex64, device="cuda", generator=g)
    dC = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")

    def stride(ls, l):
        return 1 << (len(ls) - 1 - ls.index(l))

    ms = rng.integers(0, 1 << nm, 64)
    ns = rng.integers(0, 1 << nn, 64)
    ks = np.arange(1 << nk)

    def offsets(ls, idx, bits):
        o = np.zeros(len(idx), dtype=np.int64)
        for i, l in enumerate(bits):
            o += ((idx >> i) & 1) * stride(ls, l)
        return o

    a_rows = offsets(la, ms, M)[:, None] + offsets(la, ks, K)[None, :]
    b_cols = offsets(lb, ks, K)[None, :] + offsets(lb, ns, N)[:, None]
    A_s = dA[torch.from_numpy(a_rows).cuda()].cpu().numpy().astype(np.complex128)
    B_s = dB[torch.from_numpy(b_cols).cuda()].cpu().numpy().astype(np.complex128)
    ref = np.sum(A_s * B_s, axis=1)
    c_off = torch.from_numpy(offsets(lc, ms, M) + offsets(lc, ns, N)).cuda()
    for precision, algo, tol in (("split_bf16", "fused_tc", 1e-4), ("c64", "fused_simt", 1e-5)):
        T.contract_pair(dA, la, dB, lb, dC, lc, precision=precision, algo=algo)
        torch.cuda.synchronize()
        got = dC[c_off].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (algo, np.linalg.norm(got - ref) / np.linalg.norm(ref))
    del dA, dB, dC
    torch.cuda.empty_cache()


@pytest.mark.parametrize("nm,nn,nk", [(9, 7, 6), (12, 8, 9), (14, 7, 5)])
@pytest.mark.parametrize("precision", ["split_bf16", "split_fp16"])
def test_output_layout_interleaving_rows_and_columns(nm, nn, nk, precision):
    """An output whose fastest indices alternate between the GEMM's row and
    column indices (stride 1 a row index, strides 2, 4, 8 column indices):
    the chunked kernel stages each warp's sub-tile in shared memory in the
    output's own order and stores contiguous runs.  Against FP64 einsum."""
    T = tnlib()
    import torch
    M, N, K = list(range(nm)), list(range(nm, nm + nn)), list(range(nm + nn, nm + nn + nk))
    la, lb = M + K, N + K                      # row bit 0 = M[-1], column bit j = N[-1 - j]
    fast = [N[-3], N[-2], N[-1], M[-1]]        # C's four fastest indices, slowest of them first
    lc = [x for x in M + N if x not in fast] + fast
    A = I.random_tensor(len(la), 61).astype(np.complex64)
    B = I.random_tensor(len(lb), 62).astype(np.complex64)
    sub = lambda ls: "".join(LETTERS[x] for x in ls)
    ref = np.einsum(f"{sub(la)},{sub(lb)}->{sub(lc)}", A.astype(np.complex128).reshape((2,) * len(la)),
                    B.astype(np.complex128).reshape((2,) * len(lb))).reshape(-1)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((1 << len(lc),), float("nan"), dtype=torch.complex64, device="cuda")
    T.contract_pair(dA, la, dB, lb, dC, lc, precision=precision, algo="fused_tc")
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.complex128)
    assert np.isfinite(got).all()
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
