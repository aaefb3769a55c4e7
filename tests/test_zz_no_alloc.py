"""The no-allocation tensor-train entry point against cbc_apply.

cbc_apply_tt_noalloc serves callers that may not allocate device memory when they
need an application (their framework owns all device memory through its own pool, or
their host loop forbids allocation after start-up): it keeps every intermediate in a
fixed scratch array inside the library and writes the result into a buffer the caller
owns.  This test feeds it device inputs, calls it twice in a row on the same inputs,
and requires each result to match cbc_apply (the entry point that allocates) within
the FP64 bar of the other parity tests.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

from oracle import metrics
from synth import make_problem

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10


def _noalloc(prob):
    import torch

    from paper_2601_19650_gb300 import _cbc

    st, op = prob.state, prob.op
    cplx = np.iscomplexobj(st.tensors[0])
    tdt = torch.complex128 if cplx else torch.float64
    dev_st = [torch.from_numpy(t).to("cuda").to(tdt).contiguous() for t in st.tensors]
    dev_op = [torch.from_numpy(t).to("cuda").to(tdt).contiguous() for t in op.tensors]
    cap = 1 << 20
    out = torch.zeros(cap, dtype=tdt, device="cuda")
    torch.cuda.synchronize()
    offs, bonds, log_norm = _cbc.cbc_apply_tt_noalloc(
        st.phys, st.bond, op.bond, _cbc.CBC_C128 if cplx else _cbc.CBC_F64,
        [t.data_ptr() for t in dev_st], [t.data_ptr() for t in dev_op], prob.max_bond, prob.tol,
        out.data_ptr(), cap)
    host = out.cpu().numpy()
    shape = _cbc.output_shape_fn(st.parent, st.phys)
    tens = []
    for i in range(len(st.parent)):
        shp = shape(i, bonds)
        n = int(np.prod(shp))
        tens.append(host[offs[i]: offs[i] + n].reshape(shp).copy())
    return tens, bonds, log_norm


@pytest.mark.parametrize("cfg", [
    dict(L=10, chi=16, D=4, max_bond=12, seed=3),
    dict(L=8, chi=8, D=4, max_bond=8, dtype=np.float64, seed=0),
])
def test_noalloc_matches_cbc_apply_twice(cfg):
    p = make_problem(2, **cfg)
    ref, ref_bonds, ref_log = run_gpu(p)
    for _ in range(2):
        got, bonds, log_norm = _noalloc(p)
        assert list(bonds) == list(ref_bonds)
        e = metrics.rel_err(p.state.parent, got, ref, log_norm, ref_log)
        assert e <= FP64_BAR, e


def test_noalloc_rejects_oversized_chain():
    from paper_2601_19650_gb300 import _cbc
    p = make_problem(2, L=40, chi=256, D=32, max_bond=256, dtype=np.complex128)
    st, op = p.state, p.op
    with pytest.raises(_cbc.CBCError) as ei:
        # sizes are checked before any pointer is touched or any kernel launched
        _cbc.cbc_apply_tt_noalloc(st.phys, st.bond, op.bond, _cbc.CBC_C128,
                                  [1] * len(st.phys), [1] * len(st.phys), 256, 0.0, 1, 1)
    assert ei.value.code == 1 and "scratch" in str(ei.value)
