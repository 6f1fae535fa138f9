"""The CPU oracle against facts that do not come from it (CPU only)."""
import pytest

import oracle
from oracle_checks import ALL_CHECKS


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(oracle.load())


def test_precision_barely_changes_iteration_count():
    # Section IV, Table I: 328 (double, CPU) vs 324 (single, C870) vs 323
    # (double, GTX 280) iterations on the paper's matrix, a spread of ~1.5%.
    # The same comparison on the paper-size stand-in at a loose tolerance.
    import json
    import os

    import numpy as np

    import femgen

    t1 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_table1.json")))["table1"]
    its = t1["cg_iterations"]
    paper_spread = (max(its) - min(its)) / min(its)
    s = femgen.build_system(femgen.PAPER_SIZE)
    u = s.upper()
    r64 = oracle.cg("sym", *u, s.b, tol=1e-4)
    _, it32, bd = oracle.cg_f32("sym", u[0], u[1], u[2].astype(np.float32), s.b.astype(np.float32), 1e-4, 10**5)
    assert not bd
    assert abs(it32 - r64.iterations) / r64.iterations <= max(0.05, 2 * paper_spread)
