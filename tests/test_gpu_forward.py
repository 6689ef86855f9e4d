"""Forward energy on the GPU (planes, search, full carve) against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2410_21207_gb300 import binding as sc
from paper_2410_21207_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("C", [1, 3, 4])
def test_forward_planes(dev, C):
    rng = np.random.default_rng(50 + C)
    for H, W in [(1, 1), (1, 5), (5, 1), (2, 2), (17, 33), (64, 257), (300, 1001)]:
        img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        got = sc.forward_costs(_t(img, dev))
        sc.check()
        for g, r in zip(got, oracle.forward_costs(img)):
            np.testing.assert_array_equal(g.cpu().numpy(), r, err_msg=f"{H}x{W}x{C}")


@pytest.mark.parametrize("H,W", [(1, 1), (1, 300), (5, 3), (16, 17), (63, 97), (65, 256), (129, 1000), (200, 1920),
                                 (300, 2049), (40, 4096), (1080, 64), (2000, 40)])
def test_find_seam_forward_parity(dev, H, W):
    rng = np.random.default_rng(H * 31 + W)
    for kind in ("image", "ties", "random"):
        if kind == "image":
            planes = oracle.forward_costs(rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8))
        elif kind == "ties":
            planes = oracle.forward_costs(rng.integers(0, 2, size=(H, W, 3)).astype(np.uint8))
        else:   # arbitrary planes, including nonzero entries the recurrence never uses
            planes = tuple(rng.integers(0, 700, size=(H, W)).astype(np.uint16) for _ in range(3))
        seam, cost = sc.find_seam_forward(*[_t(p, dev) for p in planes])
        sc.check()
        s_ref, c_ref = oracle.dp_seam_forward(*planes)
        assert int(cost.cpu()[0]) == c_ref, (H, W, kind)
        np.testing.assert_array_equal(seam.cpu().numpy(), s_ref, err_msg=f"{H}x{W} {kind}")


@pytest.mark.parametrize("H,W", [(2000, 300), (8192, 40), (1080, 1920)])
def test_find_seam_forward_wide_costs(dev, H, W):
    """Caller planes whose seam sums do not fit the 24-bit cost field (H * max(CU + max(DL, DR))
    >= 2^24) go to the wide-cost search; seam and cost equal the oracle's."""
    rng = np.random.default_rng(H + W)
    planes = (rng.integers(30000, 65536, size=(H, W)).astype(np.uint16),
              rng.integers(0, 65536, size=(H, W)).astype(np.uint16),
              rng.integers(0, 65536, size=(H, W)).astype(np.uint16))
    seam, cost = sc.find_seam_forward(*[_t(p, dev) for p in planes])
    sc.check()
    s_ref, c_ref = oracle.dp_seam_forward(*planes)
    assert int(cost.cpu()[0]) == c_ref
    np.testing.assert_array_equal(seam.cpu().numpy(), s_ref)


def test_carve_forward_small_both_passes(dev):
    rng = np.random.default_rng(77)
    for k in range(14):
        H, W = int(rng.integers(1, 70)), int(rng.integers(1, 120))
        C = int(rng.choice([1, 3, 4]))
        tw, th = int(rng.integers(1, W + 1)), int(rng.integers(1, H + 1))
        hi = 3 if k % 3 == 0 else 256
        img = rng.integers(0, hi, size=(H, W, C)).astype(np.uint8)
        out, log, cost = sc.carve_forward(_t(img, dev), tw, th, with_log=True)
        sc.check()
        r_out, r_log, r_cost = oracle.carve_forward(img, tw, th, with_log=True)
        np.testing.assert_array_equal(log.cpu().numpy(), r_log)
        np.testing.assert_array_equal(cost.cpu().numpy(), r_cost)
        np.testing.assert_array_equal(out.cpu().numpy(), r_out)


def test_carve_forward_generated(dev):
    img = synth.gen_image(480, 270, 6, 20, 120, 909)
    out, log, cost = sc.carve_forward(_t(img, dev), 360, 240, with_log=True)
    sc.check()
    r_out, r_log, r_cost = oracle.carve_forward(img, 360, 240, with_log=True)
    np.testing.assert_array_equal(log.cpu().numpy(), r_log)
    np.testing.assert_array_equal(out.cpu().numpy(), r_out)


def test_forward_width_limit(dev):
    with pytest.raises(sc.ScError):
        sc.carve_forward(torch.zeros((8, 5000, 3), dtype=torch.uint8, device=dev), 4990, 8)
