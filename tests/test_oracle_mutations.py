"""Plant plausible mistakes in a copy of the oracle and check that a pin catches each.

The copy is built from the oracle's source text with one substitution and executed as
a fresh module on the CPU; the real oracle is never modified.
"""
import importlib.util
import os
import sys
import types

import pytest

from pins import ALL_CHECKS

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "oracle", "cbc.py")

MUTATIONS = {
    "tt-R-update-drops-conj": ('Q.conj(), Z', 'Q, Z'),
    "tt-forward-output-legs-transposed": ('"xbsA,bPsB->xPAB"', '"xbsA,bPsB->xPBA"'),
    "tt-forward-operator-in-out-swapped": ('"xbsA,bPsB->xPAB"', '"xbsA,bsPB->xPAB"'),
    "tt-backward-operator-in-out-swapped": ('"asyB,bPsB->abPy"', '"asyB,bsPB->abPy"'),
    "compress-drops-singular-values": ('s[:k, None] * Vh[:k, :]', 'Vh[:k, :]'),
    "compress-keeps-smallest": ('s[:k, None] * Vh[:k, :]', 's[-k:, None] * Vh[-k:, :]'),
    "tol-rule-not-squared": ('tail <= tol * tol * tail[0]', 'tail <= tol * tail[0]'),
    "rank-ignores-max-bond": ('k = min(k, int(max_bond))', 'k = k'),
    "tree-R-update-drops-conj": ('Q.conj(), [_X_NEW', 'Q, [_X_NEW'),
    "tree-step2-excludes-wrong-child": ('if c != k:\n                    ops', 'if c == k:\n                    ops'),
    "tree-step3-env-from-step1": ('env_ops = [Ldown[i], [_X_P, _A_P, _B_P]]',
                                  'env_ops = [Lsub.get(i, Ldown[i]), [_X_P, _A_P, _B_P]]'),
    "lq-uses-transpose-not-adjoint": ('np.linalg.qr(S.conj().T, mode="reduced")',
                                      'np.linalg.qr(S.T, mode="reduced")'),
    # caught only by the dense-Gram pin on branching trees (isometries, projection and
    # exactness still hold: the truncation just keeps a worse subspace)
    "tree-step1-child-env-conjugated": (
        '            ops += [Lsub[c], [_x(j), _a(j), _b(j)]]\n        out_legs = [_S_OUT]',
        '            ops += [Lsub[c].conj(), [_x(j), _a(j), _b(j)]]\n        out_legs = [_S_OUT]'),
    "tree-step2-sibling-env-conjugated": (
        'if c != k:\n                    ops += [Lsub[c], ',
        'if c != k:\n                    ops += [Lsub[c].conj(), '),
}


def _mutant(name, old, new):
    src = open(ORACLE).read()
    assert src.count(old) >= 1, f"mutation {name}: pattern not found"
    src = src.replace(old, new)
    modname = f"oracle_mutant_{name.replace('-', '_')}"
    mod = types.ModuleType(modname)
    sys.modules[modname] = mod          # dataclasses resolve annotations through it
    exec(compile(src, f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name):
    old, new = MUTATIONS[name]
    mod = _mutant(name, old, new)
    caught = []
    for check in ALL_CHECKS:
        try:
            check(mod)
        except Exception as e:  # an assertion, or a shape error the mistake causes
            caught.append((check.__name__, type(e).__name__))
    assert caught, f"no pin caught mutation {name}"
