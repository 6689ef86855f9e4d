"""Parity of sc_find_seam_multi (n maps of one size searched in one launch, one cluster per map)
with the oracle's Algorithm 3 seam of each map, including full 3840 x 2160 maps."""
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


def _maps(rng, n, H, W):
    kinds = [
        lambda: rng.integers(0, 1531, size=(H, W)),
        lambda: rng.integers(0, 3, size=(H, W)),                 # many exact ties
        lambda: np.full((H, W), 5),                              # constant: leftmost straight seam
        lambda: np.tile(rng.integers(0, 40, size=(1, W)), (H, 1)),
    ]
    return [kinds[k % len(kinds)]().astype(np.uint16) for k in range(n)]


def _check(dev, maps):
    got_s, got_c = sc.find_seam_multi([torch.from_numpy(m).to(dev) for m in maps])
    sc.check()
    got_s, got_c = got_s.cpu().numpy(), got_c.cpu().numpy()
    for k, m in enumerate(maps):
        s_ref, c_ref = oracle.dp_seam(m)
        assert int(got_c[k]) == c_ref, k
        np.testing.assert_array_equal(got_s[k], s_ref, err_msg=f"map {k} of {len(maps)}, {m.shape}")


SHAPES = [(8, 8), (8, 16), (4, 8), (4, 16)]   # (compute warps per CTA, DP tile rows)
OWN_COLS = {(8, 8): 768, (8, 16): 640, (4, 8): 320, (4, 16): 256}   # columns each CTA owns


@pytest.fixture
def shape(request):
    sc.find_seam_multi_shape(*request.param)
    yield request.param
    sc.find_seam_multi_shape(0, 0)


@pytest.mark.parametrize("shape", SHAPES, indirect=True)
@pytest.mark.parametrize("H,W,n", [(1, 1, 1), (1, 300, 3), (17, 96, 4), (65, 257, 5), (130, 700, 7),
                                   (300, 2049, 3), (200, 3840, 6), (64, 8192, 2), (2000, 40, 3)])
def test_multi_parity(dev, shape, H, W, n):
    if OWN_COLS[shape] * 16 < W:
        with pytest.raises(sc.ScError):
            sc.find_seam_multi([torch.zeros((H, W), dtype=torch.uint16, device=dev)])
        return
    rng = np.random.default_rng(H * 131 + W * 7 + n)
    _check(dev, _maps(rng, n, H, W))


def test_multi_shape_rejected():
    with pytest.raises(sc.ScError):
        sc.find_seam_multi_shape(5, 8)


def test_multi_equals_single(dev):
    rng = np.random.default_rng(5)
    maps = [torch.from_numpy(m).to(dev) for m in _maps(rng, 9, 333, 1500)]
    s_multi, c_multi = sc.find_seam_multi(maps)
    for k, m in enumerate(maps):
        s1, c1 = sc.find_seam(m)
        assert torch.equal(s_multi[k], s1) and int(c_multi[k]) == int(c1[0])
    sc.check()


@pytest.mark.parametrize("shape", SHAPES + [(0, 0)], indirect=True)
def test_multi_uhd(dev, shape):
    """Full 3840 x 2160 maps: the energy of the 4K synthetic image, its mirror, and two random maps."""
    job = synth.config3()
    e = oracle.energy(job.make())
    rng = np.random.default_rng(2160)
    maps = [e.astype(np.uint16), np.ascontiguousarray(e[:, ::-1]).astype(np.uint16)] + _maps(rng, 2, 2160, 3840)
    _check(dev, maps)


@pytest.mark.parametrize("W", [904, 900])
def test_multi_range_boundary(dev, W):
    """The 24-bit range check at its exact boundary, H * max(e) = 2^24 - 1 (fast search) against
    2^24 (wide-cost search), for maps read in place (W a multiple of 8) and maps that are copied
    first (W = 900, and a map whose base is not 16-byte aligned); every seam and cost equals the
    oracle's."""
    H = 1024
    rng = np.random.default_rng(W)
    lim = ((1 << 24) - 1) // H          # 16383: the largest energy the 24-bit search takes at H = 1024
    maps = []
    for top in (lim, lim + 1):
        m = rng.integers(0, top, size=(H, W)).astype(np.uint16)
        m[rng.integers(0, H), rng.integers(0, W)] = top   # one cell at the boundary value
        maps.append(m)
    maps.append(np.full((H, W), lim + 1, dtype=np.uint16))
    _check(dev, maps)
    # a map whose rows start 2 bytes past a 16-byte boundary (a view into a larger buffer)
    buf = torch.from_numpy(np.concatenate([np.zeros(1, np.uint16), maps[1].ravel()])).to(dev)
    view = buf[1:].view(H, W)
    got_s, got_c = sc.find_seam_multi([view, torch.from_numpy(maps[0]).to(dev)])
    sc.check()
    for k, m in enumerate([maps[1], maps[0]]):
        s_ref, c_ref = oracle.dp_seam(m)
        assert int(got_c[k]) == c_ref
        np.testing.assert_array_equal(got_s[k].cpu().numpy(), s_ref)


def test_multi_mixed_energy_ranges(dev):
    """Maps of one batch on both sides of the 24-bit cost limit: each map's range is checked on its
    own, the over-range ones go to the wide-cost search, and every seam and cost equals the
    oracle's."""
    rng = np.random.default_rng(90)
    H, W = 1200, 904
    maps = [rng.integers(0, 1531, size=(H, W)), np.full((H, W), 65535), rng.integers(0, 65536, size=(H, W)),
            rng.integers(0, 3, size=(H, W)), rng.integers(65530, 65536, size=(H, W)), np.full((H, W), 9)]
    _check(dev, [m.astype(np.uint16) for m in maps])
    # the tallest over-range maps, twice in a row (the second call reuses the scratch)
    for _ in range(2):
        _check(dev, [np.full((8192, 40), 60000, dtype=np.uint16),
                     rng.integers(0, 65536, size=(8192, 40)).astype(np.uint16)])
