"""The kernels' bounded mbarrier wait (every wait of the sweep kernels gives up after a time
limit instead of spinning): on a barrier that was arrived at it completes at once; on one that
nothing arrives at it gives up after its limit with the timeout status and the abort flag set,
the kernel returns, and the context stays usable for a solve.  Nothing here faults or hangs
the GPU: the wait is bounded by the global timer."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_wait_completes_when_arrived():
    from paper_1701_04900_gb300 import native
    rc, done, err, abort, us = native.wait_check(True, 50_000_000)
    assert (rc, done, err, abort) == (native.OK, 1, 0, 0)
    assert us < 50_000


def test_wait_runs_out_and_context_stays_usable():
    import torch
    from paper_1701_04900_gb300 import native, Solver
    rc, done, err, abort, us = native.wait_check(False, 20_000_000)
    assert (rc, done, err, abort) == (native.ETIMEOUT, 0, native.ETIMEOUT, 1)
    assert 20_000 <= us < 2_000_000
    # the context still runs kernels: a small solve to its tolerance
    rng = np.random.default_rng(3)
    m, n = 300, 200
    At = torch.from_numpy((rng.standard_normal((n, m)) / np.sqrt(m)).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal(m).astype(np.float32)).cuda()
    s = Solver(At, b, 0.1, m=m, mode="async", num_ctas=1, max_sweeps=3000)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = s.solve(x)
    s.close()
    assert st["status"] == native.OK and st["stat_xhat"] <= 1e-5


def test_wait_check_rejects_bad_limits():
    from paper_1701_04900_gb300 import native
    for lim in (0, 999, 2_000_000_000):
        with pytest.raises(native.AsyflexaError):
            native.wait_check(False, lim)
