"""sc_find_seam_static, the seam search for callers that must not allocate device memory (its
scratch is a fixed array inside the library): through the C ABI it must return exactly what
sc_find_seam returns, on two calls in a row. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2410_21207_gb300 import binding as sc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    return torch.device("cuda:0")


def _pair(dev, e_np):
    e = torch.from_numpy(e_np).to(dev)
    s_ref, c_ref = sc.find_seam(e)
    sc.check()
    s_fix, c_fix = sc.find_seam_static(e)
    torch.cuda.synchronize()
    return s_ref.cpu().numpy(), int(c_ref.cpu()[0]), s_fix.cpu().numpy(), int(c_fix.cpu()[0])


def test_static_scratch_search_matches_allocating_search(dev):
    rng = np.random.default_rng(77)
    # two calls in a row: a large map, then a smaller one with many ties (the second call sees
    # the first call's leftovers in the shared array)
    maps = [rng.integers(0, 1531, size=(1080, 1920)).astype(np.uint16),
            rng.integers(0, 3, size=(333, 700)).astype(np.uint16)]
    for e_np in maps:
        s_ref, c_ref, s_fix, c_fix = _pair(dev, e_np)
        np.testing.assert_array_equal(s_fix, s_ref)   # integer path: exact
        assert c_fix == c_ref


def test_static_scratch_limits(dev):
    e = torch.zeros((4000, 4000), dtype=torch.uint16, device=dev)   # needs more than the array holds
    with pytest.raises(sc.ScError):
        sc.find_seam_static(e)
    # energies that could overflow the 24-bit cost field: the search is refused through the outputs
    big = torch.full((2000, 16), 60000, dtype=torch.uint16, device=dev)
    seam, cost = sc.find_seam_static(big)
    torch.cuda.synchronize()
    assert int(cost.cpu()[0]) == -1 and bool((seam == -1).all())
