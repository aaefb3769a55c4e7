"""The library's truncation rank rule (host code of the C ABI, no GPU) against the oracle's.

Both follow the same rule (Sec. III A compression to a bond cap, Sec. V tolerance): the
singular values above the rank floor, then the smallest rank whose relative discarded
weight is within tol^2, then the cap.  The library decides on weights w_j = s_j^2, the
oracle on the singular values; on spectra of every shape (flat, graded, with gaps, with
values below the floor) both must keep the same rank and report the same discarded weight.
"""
import numpy as np
import pytest

from oracle import cbc as oracle_cbc
from paper_2601_19650_gb300 import _cbc, build

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _spectra():
    rng = np.random.default_rng(5)
    out = [np.sort(rng.uniform(0.1, 1.0, 40))[::-1],               # flat
           np.logspace(0, -14, 60),                                # graded past the floor
           np.concatenate([np.ones(8), 1e-3 * np.ones(8), 1e-9 * np.ones(8)]),
           np.array([1.0]),
           np.concatenate([np.logspace(0, -6, 30), np.zeros(5)])]
    for _ in range(20):
        n = int(rng.integers(1, 80))
        out.append(np.sort(np.exp(rng.normal(0, 4, n)))[::-1])
    return out


@pytest.mark.parametrize("max_bond", [0, 1, 7, 32])
@pytest.mark.parametrize("tol", [0.0, 1e-1, 1e-3, 1e-8])
def test_rank_rule_matches_oracle(max_bond, tol):
    for s in _spectra():
        k_ref = oracle_cbc.choose_rank(s, max_bond, tol, oracle_cbc.EPS_RANK)
        k, disc = _cbc.cbc_rank_rule(s ** 2, 0.0, max_bond, tol, oracle_cbc.EPS_RANK)
        assert k == k_ref, (s[:5], s.size, max_bond, tol, k, k_ref)
        ref_disc = float(np.sum(s[k_ref:] ** 2) / np.sum(s ** 2))
        assert abs(disc - ref_disc) <= 1e-12 * max(ref_disc, 1e-300) + 1e-300, (disc, ref_disc)


def test_weight_beyond_the_candidates_counts_for_the_tolerance():
    # four candidates carry 99% of the weight; the 1% outside them forces k = 4 at tol 0.05
    # (0.01 > 0.05^2) but allows k = 2 at tol 0.5
    w = np.array([0.5, 0.3, 0.15, 0.04])
    assert _cbc.cbc_rank_rule(w, 0.01, 0, 0.05, 1e-12)[0] == 4
    k, disc = _cbc.cbc_rank_rule(w, 0.01, 0, 0.5, 1e-12)
    assert k == 2 and abs(disc - 0.2) < 1e-12


def test_rank_rule_rejects_bad_arguments():
    with pytest.raises(_cbc.CBCError):
        _cbc.cbc_rank_rule(np.zeros(0), 0.0, 0, 0.0, 1e-12)
    with pytest.raises(_cbc.CBCError):
        _cbc.cbc_rank_rule(np.ones(3), 0.0, 0, float("nan"), 1e-12)
