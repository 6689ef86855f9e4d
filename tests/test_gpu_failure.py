"""Failure detection without a GPU fault: a bounded device wait that nothing completes runs out,
the kernel records a timeout and returns, sc_check reports SC_ETIMEOUT, and the context stays
usable (the error word is cleared and the next search is exact)."""
import numpy as np
import pytest

import oracle
from paper_2410_21207_gb300 import binding as sc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    return torch.device("cuda:0")


def test_bounded_wait_times_out_and_context_survives(dev):
    sc.check()
    sc.selftest_wait_timeout(2000)   # 2 ms
    with pytest.raises(sc.ScError) as ei:
        sc.check()
    assert ei.value.code == sc.SC_ETIMEOUT
    sc.check()   # the error word was cleared
    e = np.random.default_rng(3).integers(0, 1531, size=(300, 700)).astype(np.uint16)
    seam, cost = sc.find_seam(torch.from_numpy(e).to(dev))
    sc.check()
    s_ref, c_ref = oracle.dp_seam(e)
    assert int(cost.cpu()[0]) == c_ref
    np.testing.assert_array_equal(seam.cpu().numpy(), s_ref)


def test_selftest_limit_checked(dev):
    with pytest.raises(sc.ScError):
        sc.selftest_wait_timeout(0)


def test_check_on_fresh_streams_reports_nothing(dev):
    """sc_check on a stream that never ran library work: its flag words are created zeroed, so
    whatever the freshly allocated device memory held is not read as an error."""
    junk = torch.full((1 << 22,), 0x5A, dtype=torch.uint8, device=dev)
    del junk
    torch.cuda.empty_cache()
    for _ in range(4):
        s = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s):
            sc.check()
