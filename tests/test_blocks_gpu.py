"""Kernel-level tests of the FP64 stages through the C ABI building blocks.

* cbc_heev (the truncation eigensolver): residual ||A U - U diag(lam)||, orthonormality
  of U and the eigenvalues against numpy's, at m = 256, 960 (the global-memory reduction
  and Cholesky panel sizes) and 4096 (config 5's Gram matrices), in FP64 and with the
  mixed path's double-float reduction for batches.
* cbc_cholqr2 (the LQ of the backward sweep): orthonormal rows, the same row space as S,
  S Q^H lower triangular with a positive diagonal (the Cholesky factor), and a clean
  CBC_ERR_NOT_POSITIVE_DEFINITE for a rank-deficient S.
* the library's Newton reciprocal and reciprocal square root against correctly rounded
  values over the whole exponent range (and against CUDA's 1.0 / x and rsqrt).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    import torch

    from paper_2601_19650_gb300 import _cbc
    return torch, _cbc


def _hermitian(m, cplx, seed, spectrum=None):
    rng = np.random.default_rng([seed, 77])
    if spectrum is None:
        x = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cplx else 0)
        return (x + x.conj().T) / 2
    # a prescribed spectrum: A = Q diag(spectrum) Q^H with Q from a Householder product
    a = np.diag(spectrum).astype(np.complex128 if cplx else np.float64)
    for _ in range(3):
        v = rng.standard_normal(m) + (1j * rng.standard_normal(m) if cplx else 0)
        v /= np.linalg.norm(v)
        h = np.eye(m) - 2 * np.outer(v, v.conj())
        a = h @ a @ h.conj().T
    return (a + a.conj().T) / 2


@pytest.mark.parametrize("m,kmax,cplx,nb,mixed", [
    (256, 128, True, 1, False), (256, 128, True, 4, True), (256, 256, False, 2, False),
    (960, 480, True, 1, False), (960, 240, True, 3, True), (4096, 1024, True, 1, False)])
def test_heev_residual_orthogonality_eigenvalues(m, kmax, cplx, nb, mixed):
    torch, c = _lib()
    mats = [_hermitian(m, cplx, seed=s) for s in range(nb)]
    tdt = torch.complex128 if cplx else torch.float64
    A = torch.from_numpy(np.stack(mats)).to("cuda", tdt).contiguous()
    lam = torch.zeros(nb, m, dtype=torch.float64, device="cuda")
    U = torch.zeros(nb, m, kmax, dtype=tdt, device="cuda")
    c.cbc_heev(c.CBC_C128 if cplx else c.CBC_F64, m, kmax, nb, A.data_ptr(), lam.data_ptr(),
               U.data_ptr(), mixed)
    lam_h, U_h = lam.cpu().numpy(), U.cpu().numpy()
    # double-float reduction: ~2^-46 per operation instead of 2^-53
    tol = (3e-11 if mixed else 2e-12) * max(1.0, m / 256) ** 0.5
    for b, a in enumerate(mats):
        ref = np.linalg.eigvalsh(a)[::-1]
        scale = np.abs(ref).max()
        l, u = lam_h[b, :kmax], U_h[b]
        assert np.abs(l - ref[:kmax]).max() <= tol * scale, np.abs(l - ref[:kmax]).max() / scale
        res = np.linalg.norm(a @ u - u * l, axis=0).max() / scale
        assert res <= tol * 10, res
        orth = np.abs(u.conj().T @ u - np.eye(kmax)).max()
        assert orth <= tol * 10, orth


def test_heev_clustered_spectrum():
    """Eigenvalues in clusters 1e-9 apart (inside the solver's cluster tolerance): the
    vectors are orthogonalised within each cluster, so U stays orthonormal and spans the
    right invariant subspace.  Inside a cluster an individual vector is any mix of its
    members, so the residual is checked on the subspace (A U = U (U^H A U)) and the
    eigenvalues as the Ritz values of U^H A U."""
    torch, c = _lib()
    m, kmax = 256, 96
    rng = np.random.default_rng(5)
    base = np.sort(rng.uniform(0.1, 1.0, m // 4))[::-1]
    spec = np.repeat(base, 4) + np.tile(np.arange(4) * 1e-9, m // 4)
    spec = np.sort(spec)[::-1]
    a = _hermitian(m, True, 9, spec)
    A = torch.from_numpy(a).to("cuda").contiguous()
    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    U = torch.zeros(m, kmax, dtype=torch.complex128, device="cuda")
    c.cbc_heev(c.CBC_C128, m, kmax, 1, A.data_ptr(), lam.data_ptr(), U.data_ptr(), False)
    u, l = U.cpu().numpy(), lam.cpu().numpy()[:kmax]
    assert np.abs(u.conj().T @ u - np.eye(kmax)).max() < 1e-11
    h = u.conj().T @ a @ u
    assert np.linalg.norm(a @ u - u @ h, axis=0).max() < 1e-11
    ritz = np.sort(np.linalg.eigvalsh(h))[::-1]
    assert np.abs(ritz - spec[:kmax]).max() < 1e-12
    # the reported values are each vector's Rayleigh quotient: within the cluster width
    assert np.abs(l - spec[:kmax]).max() < 1e-8


@pytest.mark.parametrize("m,n,cplx,nb", [(64, 300, True, 2), (256, 2048, True, 1),
                                         (100, 101, False, 3), (480, 960, True, 1)])
def test_cholqr2_against_numpy(m, n, cplx, nb):
    torch, c = _lib()
    rng = np.random.default_rng([m, n])
    S = rng.standard_normal((nb, m, n)) + (1j * rng.standard_normal((nb, m, n)) if cplx else 0)
    tdt = torch.complex128 if cplx else torch.float64
    dS = torch.from_numpy(S).to("cuda", tdt).contiguous()
    c.cbc_cholqr2(c.CBC_C128 if cplx else c.CBC_F64, m, n, nb, dS.data_ptr())
    Q = dS.cpu().numpy()
    for b in range(nb):
        q, s = Q[b], S[b]
        assert np.abs(q @ q.conj().T - np.eye(m)).max() < 1e-13
        R = s @ q.conj().T                         # S = R Q
        assert np.linalg.norm(s - R @ q) < 1e-12 * np.linalg.norm(s)
        assert np.abs(np.triu(R, 1)).max() < 1e-12 * np.abs(R).max()
        d = np.diag(R)
        assert np.all(d.real > 0) and np.abs(d.imag).max() < 1e-12 * np.abs(d).max()
        # the same factor as numpy's QR of S^H, up to the signs of its diagonal
        _, rh = np.linalg.qr(s.conj().T)
        ph = np.diag(rh) / np.abs(np.diag(rh))
        Rn = (rh * ph.conj()[:, None]).conj().T
        assert np.abs(Rn - R).max() < 1e-10 * np.abs(R).max()


def test_cholqr2_rank_deficient_reports_status():
    torch, c = _lib()
    rng = np.random.default_rng(3)
    S = rng.standard_normal((40, 200))
    S[7] = S[3]  # two equal rows
    dS = torch.from_numpy(S).to("cuda").contiguous()
    with pytest.raises(c.CBCError) as ei:
        c.cbc_cholqr2(c.CBC_F64, 40, 200, 1, dS.data_ptr())
    assert ei.value.code == 4


def _ulp_dist(a, b):
    """distance in units in the last place between doubles of the same sign"""
    ia = a.view(np.int64).astype(object)
    ib = b.view(np.int64).astype(object)
    return np.array([abs(x - y) for x, y in zip(ia, ib)], dtype=np.float64)


def test_newton_reciprocals_over_the_exponent_range():
    torch, c = _lib()
    rng = np.random.default_rng(17)
    e = rng.integers(-1020, 1021, 20000)
    mant = rng.uniform(1.0, 2.0, e.size)
    x = np.ldexp(mant, e)
    x[::2] *= -1.0  # negative values for the reciprocal
    special = np.array([1.0, 2.0, 0.5, 3.0, 1.0 / 3.0, 2.2250738585072014e-308,
                        1.7976931348623157e308, 4.9e-324, 1e-310, 1e-300, 1e300, 7.0,
                        np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)])
    x = np.concatenate([x, special, -special])
    dx = torch.from_numpy(x).to("cuda")
    out = torch.zeros(4 * x.size, dtype=torch.float64, device="cuda")
    c.cbc_selftest_math(dx.data_ptr(), out.data_ptr(), x.size)
    o = out.cpu().numpy().reshape(-1, 4)
    rcp, rcp_cuda, rs, rs_cuda = o[:, 0], o[:, 1], o[:, 2], o[:, 3]
    with np.errstate(over="ignore"):
        ref = (1.0 / x.astype(np.longdouble)).astype(np.float64)
    assert np.array_equal(np.isinf(ref), np.isinf(rcp))
    fin = np.isfinite(ref) & (np.abs(ref) >= 2.2250738585072014e-308)
    assert _ulp_dist(rcp[fin], ref[fin]).max() <= 1.0
    assert np.array_equal(rcp_cuda[fin], ref[fin])  # IEEE division is correctly rounded
    # results in the subnormal range keep their absolute accuracy
    sub = np.isfinite(ref) & ~fin
    assert np.all(np.abs(rcp[sub] - ref[sub]) <= 2 * 4.9e-324)
    pos = x > 0
    ref_rs = (1.0 / np.sqrt(x[pos].astype(np.longdouble))).astype(np.float64)
    # two Newton steps from the single-precision seed: the last step's own rounding
    # leaves at most 2 ulp, as for CUDA's rsqrt
    assert _ulp_dist(rs[pos], ref_rs).max() <= 2.0
    assert _ulp_dist(rs_cuda[pos], ref_rs).max() <= 2.0
