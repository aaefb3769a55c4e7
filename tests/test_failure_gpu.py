"""Failure detection on the GPU path, with nothing faulted, trapped or hung.

* A NaN in an input tensor is rejected when the network is created (CBC_ERR_NUMERICAL).
* An overflow inside the sweeps (inputs scaled so that the Gram's weights exceed the
  double range) is reported by cbc_apply as CBC_ERR_NUMERICAL.
* An operator that annihilates the state (all zero) gives CBC_ERR_NUMERICAL with a
  message saying that O|psi> vanishes; a rank-deficient operator is an ordinary input
  and matches the oracle.
* The bounded device-side wait every kernel uses gives up after its limit: the
  self-test waits on a word nothing writes, the kernel returns CBC_ERR_TIMEOUT, and the
  context stays usable (an application right after it succeeds).
"""
import time

import numpy as np
import pytest

from oracle import cbc as oracle_cbc
from oracle import metrics
from synth import make_problem

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


def _cbc():
    from paper_2601_19650_gb300 import _cbc as mod
    return mod


def test_nan_input_is_rejected_at_creation():
    c = _cbc()
    p = make_problem(2, L=6, chi=8, D=3, max_bond=8, dtype=np.complex128, seed=1)
    ts = [t.copy() for t in p.state.tensors]
    ts[3].flat[5] = np.nan
    with pytest.raises(c.CBCError) as ei:
        c.create_from_host(p.state.parent, p.state.phys, p.state.bond, ts, "state")
    assert ei.value.code == 5 and "NaN" in str(ei.value)
    ws = [w.copy() for w in p.op.tensors]
    ws[2].flat[0] = np.inf
    with pytest.raises(c.CBCError) as ei:
        c.create_from_host(p.op.parent, p.op.phys, p.op.bond, ws, "op")
    assert ei.value.code == 5


def test_overflow_in_the_sweep_is_reported():
    c = _cbc()
    p = make_problem(2, L=6, chi=8, D=3, max_bond=8, dtype=np.float64, seed=2)
    p.state.tensors = [t * 1e160 if i in (1, 2) else t for i, t in enumerate(p.state.tensors)]
    with pytest.raises(c.CBCError) as ei:
        run_gpu(p, precision=0)
    assert ei.value.code == 5, str(ei.value)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_operator_reports_vanishing_result(precision):
    c = _cbc()
    p = make_problem(2, L=6, chi=8, D=3, max_bond=8, dtype=np.complex128, seed=3)
    p.op.tensors = [np.zeros_like(w) for w in p.op.tensors]
    with pytest.raises(c.CBCError) as ei:
        run_gpu(p, precision=precision)
    assert ei.value.code == 5 and "vanishes" in str(ei.value)


@pytest.mark.parametrize("precision,bar", [(0, 1e-10), (1, 1e-6)])
def test_rank_deficient_operator_matches_oracle(precision, bar):
    """sigma' = 1 is never produced at sites 2 and 5: every environment past them has
    exactly half its directions at zero weight, which the rank floor removes."""
    p = make_problem(2, L=9, chi=12, D=4, max_bond=0, dtype=np.complex128, seed=4)
    for i in (2, 5):
        p.op.tensors[i] = p.op.tensors[i].copy()
        p.op.tensors[i][:, 1, :, ...] = 0.0
    got, bonds, log_norm = run_gpu(p, precision=precision)
    ref = oracle_cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, 0, 0.0)
    assert list(bonds) == list(ref.out_bonds)
    assert metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0) <= bar


def test_bounded_wait_gives_up_and_context_survives():
    c = _cbc()
    t0 = time.time()
    rc, returned = c.cbc_selftest_wait(20_000_000)  # ~10 ms at the boost clock
    dt = time.time() - t0
    assert rc == 6 and returned == 1, (rc, returned, c.cbc_last_error())
    assert "gave up" in c.cbc_last_error()
    assert dt < 30.0
    # a wait with room to spare... still finds nothing written, and still returns
    rc, returned = c.cbc_selftest_wait(0)
    assert rc == 6 and returned == 1
    # the context is intact: an application right after succeeds and matches the oracle
    p = make_problem(1, max_bond=8)
    got, bonds, log_norm = run_gpu(p)
    ref = oracle_cbc.cbc(p.state.parent, p.state.tensors, p.op.tensors, p.max_bond)
    assert metrics.rel_err(p.state.parent, got, ref.tensors, log_norm, 0.0) <= 1e-10
