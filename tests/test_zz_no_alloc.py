"""The no-allocation tensor-train entry point against cbc_apply and against the oracle.

cbc_apply_tt_noalloc serves callers that may not allocate device memory when they
need an application (their framework owns all device memory through its own pool, or
their host loop forbids allocation after start-up): it keeps every intermediate in a
fixed scratch array inside the library and writes the result into a buffer the caller
owns.  These tests feed it device inputs and require its result to match both
cbc_apply (the entry point that allocates), on two calls in a row, and the FP64
oracle, within the FP64 bar of the other parity tests; they also cover a complex
chain with a tolerance, a singular square backward step, an output buffer one element
too small, and a chain whose intermediates come close to the scratch size.  The file
is collected last.
"""
import numpy as np
import pytest

from oracle import cbc as oracle_cbc
from oracle import metrics
from synth import make_problem

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
SCRATCH_BYTES = 32 << 20


def _device_inputs(prob):
    import torch

    st, op = prob.state, prob.op
    cplx = np.iscomplexobj(st.tensors[0]) or np.iscomplexobj(op.tensors[0])
    tdt = torch.complex128 if cplx else torch.float64
    dev_st = [torch.from_numpy(np.asarray(t)).to("cuda").to(tdt).contiguous() for t in st.tensors]
    dev_op = [torch.from_numpy(np.asarray(t)).to("cuda").to(tdt).contiguous() for t in op.tensors]
    return cplx, tdt, dev_st, dev_op


def _noalloc(prob, cap=1 << 20, inputs=None):
    """One call; returns (tensors, bonds, log_norm, elements used)."""
    import torch

    from paper_2601_19650_gb300 import _cbc

    st, op = prob.state, prob.op
    cplx, tdt, dev_st, dev_op = inputs or _device_inputs(prob)
    out = torch.zeros(max(cap, 1), dtype=tdt, device="cuda")
    torch.cuda.synchronize()
    offs, bonds, log_norm = _cbc.cbc_apply_tt_noalloc(
        st.phys, st.bond, op.bond, _cbc.CBC_C128 if cplx else _cbc.CBC_F64,
        [t.data_ptr() for t in dev_st], [t.data_ptr() for t in dev_op], prob.max_bond, prob.tol,
        out.data_ptr(), cap)
    host = out.cpu().numpy()
    shape = _cbc.output_shape_fn(st.parent, st.phys)
    tens, used = [], 0
    for i in range(len(st.parent)):
        shp = shape(i, bonds)
        n = int(np.prod(shp))
        tens.append(host[offs[i]: offs[i] + n].reshape(shp).copy())
        used = max(used, int(offs[i]) + n)
    return tens, bonds, log_norm, used


def _oracle(prob):
    st, op = prob.state, prob.op
    return oracle_cbc.cbc(st.parent, st.tensors, op.tensors, prob.max_bond, prob.tol)


@pytest.mark.parametrize("cfg", [
    dict(L=10, chi=16, D=4, max_bond=12, seed=3),
    dict(L=8, chi=8, D=4, max_bond=8, dtype=np.float64, seed=0),
    dict(L=9, chi=16, D=4, max_bond=0, dtype=np.complex128, seed=4, tol=1e-3),
])
def test_noalloc_matches_cbc_apply_and_oracle_twice(cfg):
    cfg = dict(cfg)
    tol = cfg.pop("tol", 0.0)
    p = make_problem(2, tol=tol, **cfg)
    ref, ref_bonds, ref_log = run_gpu(p)
    orc = _oracle(p)
    inputs = _device_inputs(p)
    for _ in range(2):
        got, bonds, log_norm, _ = _noalloc(p, inputs=inputs)
        assert list(bonds) == list(ref_bonds) == list(orc.out_bonds)
        e = metrics.rel_err(p.state.parent, got, ref, log_norm, ref_log)
        assert e <= FP64_BAR, e
        e = metrics.rel_err(p.state.parent, got, orc.tensors, log_norm, 0.0)
        assert e <= FP64_BAR, e


def test_noalloc_singular_square_step():
    """A square S in the backward sweep that is singular (the operator never produces
    sigma' = 1 at site 4): the new tensor there is the identity, as in cbc_apply, so the
    call neither runs into a Cholesky breakdown nor leaves the FP64 bar."""
    p = make_problem(2, L=8, chi=8, D=4, max_bond=0, dtype=np.float64, seed=1)
    p.op.tensors[4] = p.op.tensors[4].copy()
    p.op.tensors[4][:, 1, :, ...] = 0.0
    ref, ref_bonds, ref_log = run_gpu(p)
    orc = _oracle(p)
    got, bonds, log_norm, _ = _noalloc(p)
    assert list(bonds) == list(ref_bonds) == list(orc.out_bonds)
    assert metrics.rel_err(p.state.parent, got, ref, log_norm, ref_log) <= FP64_BAR
    assert metrics.rel_err(p.state.parent, got, orc.tensors, log_norm, 0.0) <= FP64_BAR


def test_noalloc_output_one_element_short_then_exact():
    from paper_2601_19650_gb300 import _cbc

    p = make_problem(2, L=8, chi=8, D=4, max_bond=6, dtype=np.complex128, seed=2)
    inputs = _device_inputs(p)
    first, bonds0, log0, used = _noalloc(p, inputs=inputs)
    with pytest.raises(_cbc.CBCError) as ei:
        _noalloc(p, cap=used - 1, inputs=inputs)
    assert ei.value.code == 1
    assert "out_capacity" in str(ei.value)
    got, bonds, log_norm, used2 = _noalloc(p, cap=used, inputs=inputs)
    assert used2 == used and list(bonds) == list(bonds0)
    assert metrics.rel_err(p.state.parent, got, first, log_norm, log0) <= FP64_BAR


def test_noalloc_near_scratch_limit():
    """The longest chi=128, D=8 complex chain that fits the scratch array (about 31 of
    its 32 MiB; each site adds about 2 MiB) runs and matches the oracle; the chains
    beyond it are rejected with the size they would need."""
    from paper_2601_19650_gb300 import _cbc

    fits = None
    for L in range(24, 15, -1):
        p = make_problem(2, L=L, chi=128, D=8, max_bond=128, dtype=np.complex128, seed=7)
        try:
            res = _noalloc(p, cap=1 << 23)
        except _cbc.CBCError as e:
            assert e.code == 1 and "scratch" in str(e), str(e)
            need = [int(w) for w in str(e).split() if w.isdigit()]
            assert max(need) > SCRATCH_BYTES
            continue
        fits = (p, res)
        break
    assert fits is not None and 18 <= fits[0].state.n < 24
    p, (got, bonds, log_norm, _) = fits
    orc = _oracle(p)
    assert list(bonds) == list(orc.out_bonds)
    assert metrics.rel_err(p.state.parent, got, orc.tensors, log_norm, 0.0) <= FP64_BAR


def test_noalloc_rejects_oversized_chain():
    from paper_2601_19650_gb300 import _cbc
    p = make_problem(2, L=40, chi=256, D=32, max_bond=256, dtype=np.complex128)
    st, op = p.state, p.op
    with pytest.raises(_cbc.CBCError) as ei:
        # sizes are checked before any pointer is touched or any kernel launched
        _cbc.cbc_apply_tt_noalloc(st.phys, st.bond, op.bond, _cbc.CBC_C128,
                                  [1] * len(st.phys), [1] * len(st.phys), 256, 0.0, 1, 1)
    assert ei.value.code == 1 and "scratch" in str(ei.value)
