"""Seam insertion on the GPU (sc_enlarge) against the oracle's, byte for byte, with the mapped
seam columns."""
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


@pytest.mark.parametrize("H,W,C", [(1, 2, 1), (1, 40, 3), (5, 3, 4), (17, 33, 3), (64, 100, 1), (120, 257, 3),
                                   (200, 513, 4), (48, 2100, 3)])
def test_enlarge_parity(dev, H, W, C):
    rng = np.random.default_rng(H * 1000 + W + C)
    for kind in ("uniform", "ties"):
        img = rng.integers(0, 256 if kind == "uniform" else 3, size=(H, W, C)).astype(np.uint8)
        for k in sorted({1, max(1, W // 4), W - 1} if W <= 300 else {1, 37}):
            out, cols = sc.enlarge(torch.from_numpy(img).to(dev), W + k, with_cols=True)
            sc.check()
            r_out, r_cols = oracle.enlarge(img, W + k, with_cols=True)
            np.testing.assert_array_equal(cols.cpu().numpy()[:k], r_cols, err_msg=f"{H}x{W}x{C} k={k} {kind}")
            np.testing.assert_array_equal(out.cpu().numpy(), r_out, err_msg=f"{H}x{W}x{C} k={k} {kind}")


def test_enlarge_generated_image(dev):
    img = synth.gen_image(640, 360, 8, 20, 120, 4242)
    out = sc.enlarge(torch.from_numpy(img).to(dev), 800)
    sc.check()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.enlarge(img, 800))


def test_enlarge_rejects_bad_targets(dev):
    img = torch.zeros((10, 20, 3), dtype=torch.uint8, device=dev)
    for tw in (20, 40, 5):
        with pytest.raises(sc.ScError):
            sc.enlarge(img, tw)
