"""Host logic of the sweep-count contract (tests/sweep_contract.py): the
Poisson tail bound against scipy's, and the step check on planted counts."""
import numpy as np
import pytest

from tests import sweep_contract as C


@pytest.mark.parametrize("rate,n", [(3.3e-5, 1000), (3.3e-5, 1024000), (6.7e-2, 200), (0.0, 50)])
def test_allowed_beyond_is_the_poisson_tail(rate, n):
    stats = pytest.importorskip("scipy.stats")
    lam = C.MARGIN * rate * n
    m = C.allowed_beyond(rate, n)
    assert stats.poisson.sf(m, lam) < C.TAIL
    assert m == 0 or stats.poisson.sf(m - 1, lam) >= C.TAIL


def test_check_steps_accepts_and_rejects():
    d = np.zeros(100000, dtype=int)
    d[:5] = 1
    d[5] = 2
    C.check_steps(d, "kepler")              # one step beyond +-1 in 1e5: allowed
    d[6:60] = 2
    with pytest.raises(AssertionError):
        C.check_steps(d, "kepler")          # 55 steps beyond: far above 2 x 3.3e-5 x 1e5
    d[:] = 0
    d[0] = 5
    with pytest.raises(AssertionError):
        C.check_steps(d, "kepler")          # 5 apart: above the largest measured (4)
