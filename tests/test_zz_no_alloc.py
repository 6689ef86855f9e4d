"""sc_find_seam_static, the seam search for callers that must not allocate device memory: a
latency-critical loop that cannot absorb cudaMalloc's device synchronisation, or a host that budgets
every device byte through its own allocator. Its scratch is a fixed array inside the library.

Through the C ABI it must return exactly what sc_find_seam returns (on two calls in a row) and
Algorithm 3's seam as the oracle computes it, report device-side errors, and leave the device's
free memory unchanged. This file is collected last on purpose, so that a run that stops at the
first failure has run every other test first; it also passes alone in a fresh process."""
import ctypes

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


def _pair(dev, e_np):
    e = torch.from_numpy(e_np).to(dev)
    s_ref, c_ref = sc.find_seam(e)
    sc.check()
    s_fix, c_fix = sc.find_seam_static(e)
    sc.check()
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


@pytest.mark.parametrize("kind", ["uniform", "ties", "wide_costs", "uhd"])
def test_static_scratch_search_matches_oracle(dev, kind):
    """Algorithm 3's seam and cost from the oracle: a 1080 x 1920 map, a tie-heavy one, one whose
    seam sums exceed the fast search's 24-bit cost field, and a full 3840 x 2160 map (the largest
    size the array is stated to hold)."""
    rng = np.random.default_rng(1920)
    e_np = {"uniform": lambda: rng.integers(0, 1531, size=(1080, 1920)),
            "ties": lambda: rng.integers(0, 2, size=(1080, 1920)),
            "wide_costs": lambda: rng.integers(0, 65536, size=(1080, 1920)),
            "uhd": lambda: rng.integers(0, 1531, size=(2160, 3840))}[kind]().astype(np.uint16)
    seam, cost = sc.find_seam_static(torch.from_numpy(e_np).to(dev))
    sc.check()
    s_ref, c_ref = oracle.dp_seam(e_np)
    assert int(cost.cpu()[0]) == c_ref
    np.testing.assert_array_equal(seam.cpu().numpy(), s_ref)


def test_static_scratch_limits(dev):
    e = torch.zeros((4000, 4000), dtype=torch.uint16, device=dev)   # needs more than the array holds
    with pytest.raises(sc.ScError) as ei:
        sc.find_seam_static(e)
    assert ei.value.code == sc.SC_EINVAL and "bytes of scratch" in str(ei.value)


def test_static_device_errors_are_reported(dev):
    """The error path of a static call, driven without a fault by a bounded wait that runs out:
    the outputs are set to -1, the next sc_check reports the timeout (and clears it), and the next
    static search is exact again."""
    H = 777
    seam, cost = sc.find_seam_static_selftest(H, limit_us=2000)
    torch.cuda.synchronize()
    assert bool((seam == -1).all()) and int(cost.cpu()[0]) == -1
    with pytest.raises(sc.ScError) as ei:
        sc.check()
    assert ei.value.code == sc.SC_ETIMEOUT
    sc.check()   # reported once, then cleared
    e_np = np.random.default_rng(3).integers(0, 1531, size=(H, 500)).astype(np.uint16)
    s, c = sc.find_seam_static(torch.from_numpy(e_np).to(dev))
    sc.check()
    s_ref, c_ref = oracle.dp_seam(e_np)
    assert int(c.cpu()[0]) == c_ref
    np.testing.assert_array_equal(s.cpu().numpy(), s_ref)


def test_static_call_allocates_nothing(dev):
    """After a first call (which looks up the array's address), calls leave the device's free
    memory unchanged. The outputs are allocated before the measurement and the call is made
    through the C ABI directly, so that no allocator of the test itself runs in between."""
    lib = sc.load()
    H, W = 1080, 1920
    e = torch.from_numpy(np.random.default_rng(8).integers(0, 1531, size=(H, W)).astype(np.uint16)).to(dev)
    big = torch.from_numpy(np.random.default_rng(9).integers(0, 65536, size=(H, W)).astype(np.uint16)).to(dev)
    seam = torch.empty(H, dtype=torch.int32, device=dev)
    cost = torch.empty(1, dtype=torch.int64, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def call(m):
        rc = lib.sc_find_seam_static(ctypes.c_void_p(m.data_ptr()), H, W, ctypes.c_void_p(seam.data_ptr()),
                                     ctypes.c_void_p(cost.data_ptr()), st)
        assert rc == sc.SC_OK

    call(e)
    call(big)   # the wide-cost path too
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for m in (e, big, e):
        call(m)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0
    sc.check()
