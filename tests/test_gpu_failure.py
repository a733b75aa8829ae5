"""Failure detection without a GPU fault: a bounded device wait that nothing
completes turns into NSLI_ERR_TIMEOUT, and the handle keeps working."""
import numpy as np
import pytest

import oracle
from paper_2003_09956_gb300 import nsli, workloads

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_handle_recovers():
    from paper_2003_09956_gb300 import _build
    _build.build()
    # CTA 0 owns 4000/152 = 26 rows of 1000-column binary32 rows (4 KB): with
    # 16 rows per 64 KB slot it has two slots; slot 1 is never issued
    p = workloads.dense_system(4000, 1000, seed=71)
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"]) as s:
        assert s.inject_timeout(slot=1) == nsli.ERR_TIMEOUT
        # the context and the handle are still usable: a normal Map/Reduce
        # matches the oracle afterwards
        y, h, _ = s.map_reduce()
        n2, _ = oracle.norms2(p["A"])
        ref = oracle.map_reduce(p["A"], p["b0"], n2, p["x0"])
        assert abs(h - ref["h"]) <= 2
        assert np.linalg.norm(y - ref["y"]) <= 1e-4 * np.linalg.norm(ref["y"])
        s.iterate(3)
        s.sync()
        assert s.result()["tick"] == 3
