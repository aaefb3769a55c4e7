"""GPU parity at the large tensor-train workload's full local shapes: d = 4, MPS bond 1024,
MPO bond 32, complex64 Gaussian entries, cap 1024, on a 10-site chain (the shortest chain
whose middle bond reaches 1024 = 4^5).  The compression after site 6 keeps 1024 of 4096
directions of a 4096 x 8192 block: the 4096 x 4096 eigensolve, the global-memory
tridiagonal reduction and the 1024 x 1024 CholeskyQR of the backward sweep all run at the
sizes of the L = 100 workload.  The oracle (about a minute per run on the host) is
computed once per module; the tolerance run adds tol = 1e-8 to the cap."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from gpu_helpers import run_gpu  # noqa: E402
from oracle import cbc, metrics  # noqa: E402
from synth import make_problem  # noqa: E402

FP64_BAR, MIXED_BAR = 1e-10, 1e-6


@pytest.fixture(scope="module")
def large_case():
    p = make_problem(5, L=10, max_bond=1024)
    ref = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond, 0.0)
    return p, ref


@pytest.fixture(scope="module")
def large_tol_case():
    p = make_problem(5, L=10, max_bond=1024, tol=1e-8, seed=1)
    ref = cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond, p.tol)
    return p, ref


def _check(p, ref, precision, bar):
    got, bonds, log_norm = run_gpu(p, precision=precision)
    assert list(bonds) == list(ref.out_bonds), (bonds, ref.out_bonds)
    assert max(ref.env_ranks) == 1024
    e = metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0)
    assert e <= bar, e


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_bond_1024_cap(large_case, precision, bar):
    p, ref = large_case
    _check(p, ref, precision, bar)


@pytest.mark.parametrize("precision,bar", [(0, FP64_BAR), (1, MIXED_BAR)])
def test_bond_1024_cap_and_tol_1e8(large_tol_case, precision, bar):
    p, ref = large_tol_case
    _check(p, ref, precision, bar)
