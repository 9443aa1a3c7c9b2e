"""cl_zgemm_emu: the FP64-accurate complex GEMM behind CL_FP64_EMU (BF16
digit products on the tcgen05 tensor cores) against numpy's complex128 GEMM.

Bound.  Both results carry rounding errors: an FP64 GEMM is within
gamma_K |A||B| componentwise; the digit split truncates every operand at 2^-56
of its row / column maximum in each 32-element k chunk, and the dropped digit
products are below the same level.  Their difference is therefore held to
  |dC_ij| <= 4 K u (|A||B|)_ij + 8 K u max_k |a_ik| max_k |b_kj|,   u = 2^-53,
which a dropped digit level (2^-8 relative) or a wrong sign, index or scale
exceeds by many orders of magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _B():
    from paper_1707_08874_gb300 import binding as B
    return B


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _check(A, B, C0, got, beta, neg):
    ref = A @ B
    if neg:
        ref = -ref
    if beta:
        ref = ref + C0
    K = A.shape[1]
    bound = 4 * K * U * (np.abs(A) @ np.abs(B)) + 8 * K * U * np.abs(A).max(1, keepdims=True) * np.abs(B).max(
        0, keepdims=True)
    if beta:
        bound = bound + 2 * U * np.abs(C0)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    return (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 32, 32), (130, 33, 70), (257, 65, 1000), (64, 200, 24),
                                   (300, 96, 31), (2000, 700, 24), (24, 2112, 24)])
def test_zgemm_emu_random(M, N, K):
    rng = np.random.default_rng(M * 1000003 + N * 101 + K)
    A, B = _rand(rng, M, K), _rand(rng, K, N)
    got, st = _B().zgemm_emu(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st == 0
    _check(A, B, None, got.cpu().numpy(), False, False)


@pytest.mark.parametrize("K", [48, 32])
@pytest.mark.parametrize("beta,neg", [(1, 0), (1, 1), (0, 1)])
def test_zgemm_emu_beta_neg_strided(beta, neg, K):
    """C = beta C -/+ A B on sub-matrices of larger row-major arrays (lda > K);
    K = 32 runs the persistent single-chunk kernel, K = 48 the chunked one."""
    rng = np.random.default_rng(7 + 2 * beta + neg + K)
    M, N = 150, 40
    Abig, Bbig, Cbig = _rand(rng, M, K + 9), _rand(rng, K, N + 5), _rand(rng, M, N + 3)
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (Abig, Bbig, Cbig))
    got, st = _B().zgemm_emu(tA[:, :K], tB[:, :N], tC[:, :N], beta=bool(beta), neg=bool(neg))
    assert st == 0
    g = tC.cpu().numpy()
    _check(Abig[:, :K], Bbig[:, :N], Cbig[:, :N], g[:, :N], beta, neg)
    assert np.array_equal(g[:, N:], Cbig[:, N:])  # columns outside the product untouched


def test_zgemm_emu_dynamic_range():
    """Rows and columns scaled by 2^-60 .. 2^60 and chunks of different
    magnitude along k: per-row / per-column / per-chunk exponents keep every
    output at FP64 accuracy relative to its own scale."""
    rng = np.random.default_rng(11)
    M, N, K = 200, 70, 160
    A, B = _rand(rng, M, K), _rand(rng, K, N)
    A *= 2.0 ** rng.integers(-60, 61, size=(M, 1))
    B *= 2.0 ** rng.integers(-60, 61, size=(1, N))
    A[:, 32:64] *= 2.0 ** -20   # one k chunk much smaller than the others
    B[96:128] *= 2.0 ** 24      # one much larger
    got, st = _B().zgemm_emu(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st == 0
    _check(A, B, None, got.cpu().numpy(), False, False)


@pytest.mark.parametrize("K", [90, 20])
def test_zgemm_emu_exact_small_integers(K):
    """Gaussian integers below 2^8: every digit product is exact, so the
    result equals the exact integer product bit for bit."""
    rng = np.random.default_rng(3 + K)
    M, N = 140, 36
    A = rng.integers(-255, 256, (M, K)) + 1j * rng.integers(-255, 256, (M, K))
    B = rng.integers(-255, 256, (K, N)) + 1j * rng.integers(-255, 256, (K, N))
    got, st = _B().zgemm_emu(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st == 0
    assert np.array_equal(got.cpu().numpy(), A @ B)


def test_zgemm_emu_repeatable_and_zero():
    """Two calls give identical bits; zero operands give exact zeros."""
    rng = np.random.default_rng(5)
    A, B = _rand(rng, 129, 100), _rand(rng, 100, 33)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    g1, _ = _B().zgemm_emu(tA, tB)
    g2, _ = _B().zgemm_emu(tA, tB)
    assert torch.equal(g1, g2)
    z, st = _B().zgemm_emu(torch.zeros_like(tA), tB)
    assert st == 0 and not torch.any(z != 0)


def test_zgemm_emu_rejects_bad_arguments():
    import ctypes
    L = _B().load()
    n = ctypes.c_size_t()
    assert L.cl_zgemm_emu_workspace(0, 4, 4, ctypes.byref(n)) == _B().CL_ERR_INVALID_ARG
    assert L.cl_zgemm_emu_workspace(4, 4, 4, ctypes.byref(n)) == 0 and n.value > 0
    tA = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    work = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    args = [ctypes.c_void_p(tA.data_ptr()), 4, ctypes.c_void_p(tA.data_ptr()), 4, ctypes.c_void_p(tA.data_ptr()), 4,
            0, 0, ctypes.c_void_p(work.data_ptr())]
    # workspace one byte short
    assert L.cl_zgemm_emu(4, 4, 4, *args, n.value - 1, ctypes.c_void_p(st.data_ptr()), None) == \
        _B().CL_ERR_INVALID_ARG
    # misaligned A (8 bytes into the tensor)
    bad = [ctypes.c_void_p(tA.data_ptr() + 8)] + args[1:]
    assert L.cl_zgemm_emu(4, 4, 4, *bad, n.value, ctypes.c_void_p(st.data_ptr()), None) == _B().CL_ERR_INVALID_ARG
