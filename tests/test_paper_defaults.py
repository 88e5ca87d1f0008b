"""The library's and the oracle's defaults are the paper's tuned parameters
(tests/golden/paper_facts.json, each with its citation).  No GPU: the
default-parameter call of the C ABI is host code."""
import inspect

import pytest

from oracle.solvers import mirs, qtrunc_chebyshev
from oracle.subspace import rational_filter_shifts


def test_library_solver_defaults(golden):
    from paper_1402_2585_gb300 import ALG_ADEF2, Hdcg
    try:
        p = Hdcg.default_params()
    except (OSError, RuntimeError) as e:   # the library not built here
        pytest.skip(str(e))
    assert p.algorithm == ALG_ADEF2
    assert p.mirs_iter == golden["mirs_iterations"]["value"]
    assert p.mirs_shift == golden["mirs_shift"]["value"]
    assert p.coarse_tol == golden["coarse_inner_residual"]["value"]
    assert p.flexible == 1


def test_oracle_defaults(golden):
    sig = inspect.signature(mirs).parameters
    assert sig["n_iter"].default == golden["mirs_iterations"]["value"]
    assert sig["shift"].default == golden["mirs_shift"]["value"]
    q = inspect.signature(qtrunc_chebyshev).parameters
    assert q["order"].default == golden["chebyshev_order"]["value"]
    assert [q["lo"].default, q["hi"].default] == golden["chebyshev_interval"]["value"]
    lam = golden["rational_filter_lambda"]["value"]
    sig, _ = rational_filter_shifts(lam, lam / 3)
    assert sig == pytest.approx([lam, 4 * lam / 3, 5 * lam / 3, 2 * lam])
