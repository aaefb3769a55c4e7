"""Kernel-level tests of the dense product behind every contraction (cbc_gemm).

FP64 path: compared with numpy in FP64.  Tensor-core path (bf16 slices): compared with
numpy against the error bound of the slicing (each operand keeps ~8S-1 bits relative
to its row/column maximum), and bit-exact on integer inputs that the slices represent
exactly, which checks that every FP32 partial sum of the tensor cores is exact.
"""
import numpy as np
import pytest

from paper_2601_19650_gb300 import _cbc

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _run(prec, S, A, B, transA=False, conjA=False, transB=False, conjB=False):
    import torch
    cplx = np.iscomplexobj(A) or np.iscomplexobj(B)
    dt = np.complex128 if cplx else np.float64
    A = A.astype(dt)
    B = B.astype(dt)
    opA = A.T if transA else A
    opB = B.T if transB else B
    M, K = opA.shape
    N = opB.shape[1]
    dA, dB = _dev(A), _dev(B)
    C = torch.full((M, N), float("nan"), dtype=torch.complex128 if cplx else torch.float64,
                   device="cuda")
    _cbc.cbc_gemm(prec, S, _cbc.CBC_C128 if cplx else _cbc.CBC_F64, M, N, K, dA.data_ptr(),
                  A.shape[1], transA, conjA, dB.data_ptr(), B.shape[1], transB, conjB,
                  C.data_ptr(), N)
    torch.cuda.synchronize()
    ref = (np.conj(opA) if conjA else opA) @ (np.conj(opB) if conjB else opB)
    return C.cpu().numpy(), ref


def _rand(rng, shape, cplx):
    x = rng.standard_normal(shape)
    if cplx:
        x = x + 1j * rng.standard_normal(shape)
    return x


SHAPES = [(128, 64, 64), (300, 100, 250), (40, 700, 33), (1, 1, 1), (129, 65, 4100),
          (256, 2048, 256), (32, 16384, 32)]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_gemm(shape, cplx):
    rng = np.random.default_rng(hash(shape) % 1000)
    M, N, K = shape
    C, ref = _run(0, 0, _rand(rng, (M, K), cplx), _rand(rng, (K, N), cplx))
    assert np.abs(C - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()) * np.sqrt(K)


@pytest.mark.parametrize("S", [2, 3, 4, 5])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_gemm_error_bound(shape, cplx, S):
    rng = np.random.default_rng(7 + S)
    M, N, K = shape
    A = _rand(rng, (M, K), cplx)
    B = _rand(rng, (K, N), cplx)
    C, ref = _run(1, S, A, B)
    # each operand element is off by at most 2^(e-8S) (e: exponent of its row / column
    # maximum) and the dropped slice levels add at most S * 2^(e_a+e_b-8S-6) per term
    ea = 2.0 ** (np.floor(np.log2(np.abs(np.stack([A.real, A.imag])).max(axis=(0, 2)))) + 1)
    eb = 2.0 ** (np.floor(np.log2(np.abs(np.stack([B.real, B.imag])).max(axis=(0, 1)))) + 1)
    bound = (2 if cplx else 1) * K * np.outer(ea, eb) * 2.0 ** (-8 * S) * (3 + S * S / 2)
    err = np.abs(C - ref)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("cplx", [False, True])
def test_tc_gemm_exact_on_integer_grid(cplx):
    """Integer inputs with |x| <= 127 are one exact slice; with several chunks and a K
    split the result must equal the integer product exactly."""
    rng = np.random.default_rng(3)
    M, N, K = 200, 96, 5000
    A = rng.integers(-127, 128, (M, K)).astype(np.float64)
    B = rng.integers(-127, 128, (K, N)).astype(np.float64)
    A[:, 0] = 127.0  # every row / column reaches the same maximum exponent
    B[0, :] = 127.0
    if cplx:
        A = A + 1j * rng.integers(-127, 128, (M, K))
        B = B + 1j * rng.integers(-127, 128, (K, N))
    C, ref = _run(1, 2, A, B)
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("trans", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("conj", [(False, True), (True, False), (True, True)])
def test_tc_gemm_transpose_conj(trans, conj):
    rng = np.random.default_rng(11)
    M, N, K = 150, 90, 300
    A = _rand(rng, (K, M) if trans[0] else (M, K), True)
    B = _rand(rng, (N, K) if trans[1] else (K, N), True)
    C, ref = _run(1, 5, A, B, trans[0], conj[0], trans[1], conj[1])
    assert np.abs(C - ref).max() <= 1e-9 * np.abs(ref).max()
