"""Parity of the CUDA path (called through the C ABI) with the oracle: bit-exact energies, seams,
costs and carved images."""
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


def _to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("C", [1, 3, 4])
def test_energy_parity(dev, C):
    rng = np.random.default_rng(100 + C)
    shapes = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 17), (16, 16), (17, 33), (31, 129), (64, 257), (300, 1001)]
    for H, W in shapes:
        img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        got = _np(sc.energy(_to_dev(img, dev)))
        np.testing.assert_array_equal(got, oracle.energy(img), err_msg=f"{H}x{W}x{C}")
    sc.check()


def _energies(rng, H, W):
    yield "uniform", rng.integers(0, 1531, size=(H, W))
    yield "ties", rng.integers(0, 3, size=(H, W))
    yield "constant", np.full((H, W), 7)
    yield "stripes", np.tile(rng.integers(0, 50, size=(1, W)), (H, 1))


SEAM_SHAPES = [
    (1, 1), (1, 2), (2, 1), (1, 300), (5, 3), (16, 17), (17, 96), (63, 97), (64, 255), (65, 256), (127, 257),
    (128, 513), (129, 1000), (200, 1920), (300, 2049), (70, 3000), (40, 4096), (40, 4097), (33, 6000),
    (20, 8192), (1080, 64), (8192, 40),
]


@pytest.mark.parametrize("H,W", SEAM_SHAPES)
def test_find_seam_parity(dev, H, W):
    rng = np.random.default_rng(H * 10007 + W)
    for kind, e in _energies(rng, H, W):
        e = e.astype(np.uint16)
        seam, cost = sc.find_seam(_to_dev(e, dev))
        sc.check()
        s_ref, c_ref = oracle.dp_seam(e)
        assert int(_np(cost)[0]) == c_ref, (H, W, kind)
        np.testing.assert_array_equal(_np(seam), s_ref, err_msg=f"{H}x{W} {kind}")


@pytest.mark.parametrize("H,W", SEAM_SHAPES)
def test_greedy_seam_parity(dev, H, W):
    """Algorithm 2 on the GPU equals the oracle's greedy seam and cost (ties, edges, 1-wide maps)."""
    rng = np.random.default_rng(H * 7919 + W)
    for kind, e in _energies(rng, H, W):
        e = e.astype(np.uint16)
        seam, cost = sc.greedy_seam(_to_dev(e, dev))
        sc.check()
        s_ref, c_ref = oracle.greedy_seam(e)
        assert int(_np(cost)[0]) == c_ref, (H, W, kind)
        np.testing.assert_array_equal(_np(seam), s_ref, err_msg=f"{H}x{W} {kind}")


@pytest.mark.parametrize("H,W,kind", [
    (2000, 16, "const60000"),     # 2000 * 60000 >= 2^24: every seam sum beyond the 24-bit field
    (1080, 1920, "max"),          # every energy 65535: all ties, cost 1080 * 65535
    (1080, 1920, "uniform"),      # any uint16 value
    (1080, 1920, "ties"),         # 3 values near the top: many exact ties
    (8192, 40, "max"),            # the tallest map: cost 8192 * 65535 (2^29)
    (8192, 40, "uniform"),
    (257, 8192, "uniform"),       # the widest map
    (1, 1, "max"), (1, 5, "uniform"), (3, 1, "max"), (17, 63, "ties"), (300, 129, "band"),
])
def test_find_seam_wide_costs(dev, H, W, kind):
    """Maps whose seam sums do not fit the fast search's 24-bit cost field (H * max(e) >= 2^24):
    they go to the wide-cost search, and the seam and the int64 cost still equal Algorithm 3's
    (the oracle's, with int64 costs)."""
    rng = np.random.default_rng(H * 7 + W)
    e = {"const60000": lambda: np.full((H, W), 60000),
         "max": lambda: np.full((H, W), 65535),
         "uniform": lambda: rng.integers(0, 65536, size=(H, W)),
         "ties": lambda: rng.integers(65533, 65536, size=(H, W)),
         "band": lambda: rng.integers(60000, 60003, size=(H, W))}[kind]().astype(np.uint16)
    # most of these exceed the 24-bit field (H * max(e) >= 2^24); the short ones check that large
    # values that still fit stay on the fast search with the same answer
    seam, cost = sc.find_seam(_to_dev(e, dev))
    sc.check()
    s_ref, c_ref = oracle.dp_seam(e)
    assert int(_np(cost)[0]) == c_ref
    np.testing.assert_array_equal(_np(seam), s_ref)


@pytest.mark.parametrize("H,W,lo,hi", [
    (100, 1000, 0, 60000),      # energies far above any image energy
    (100, 2000, 4090, 4100),    # a narrow band of large energies (near ties)
    (3000, 300, 3000, 4095),    # tall map, costs near 2^23.5
    (4096, 200, 3800, 4095),    # costs within 2^20 of the 2^24 cost limit
    (64, 129, 4094, 4095),      # one value everywhere: all ties
])
def test_find_seam_large_costs(dev, H, W, lo, hi):
    """Maps with large energies and costs close to the 24-bit cost field's limit, several CTAs
    wide, equal to the oracle (seam and cost)."""
    rng = np.random.default_rng(H * 31 + W + lo)
    e = rng.integers(lo, hi, size=(H, W), endpoint=False).astype(np.uint16)
    seam, cost = sc.find_seam(_to_dev(e, dev))
    sc.check()
    s_ref, c_ref = oracle.dp_seam(e)
    assert int(_np(cost)[0]) == c_ref
    np.testing.assert_array_equal(_np(seam), s_ref)


def test_carve_max_energy_checkerboard(dev):
    """A 4-channel 0/255 checkerboard: every e1 energy at its maximum (2040) and ties everywhere,
    several CTAs wide, both passes."""
    H, W = 160, 700
    yy, xx = np.mgrid[0:H, 0:W]
    img = (((yy + xx) & 1) * 255).astype(np.uint8)[:, :, None].repeat(4, axis=2)
    _carve_cmp(dev, img, W - 40, H - 12)


def _carve_ref(img, tw, th):
    return oracle.carve(img, tw, th, with_log=True)


def _carve_cmp(dev, img, tw, th, plain=False):
    out, log, cost = sc.carve(_to_dev(img, dev), tw, th, with_log=True, plain=plain)
    sc.check()
    r_out, r_log, r_cost = _carve_ref(img, tw, th)
    np.testing.assert_array_equal(_np(log), r_log)
    np.testing.assert_array_equal(_np(cost), r_cost)
    np.testing.assert_array_equal(_np(out), r_out)


def test_carve_small_both_passes(dev):
    rng = np.random.default_rng(31)
    for k in range(25):
        H, W = int(rng.integers(1, 90)), int(rng.integers(1, 140))
        C = int(rng.choice([1, 3, 4]))
        tw, th = int(rng.integers(1, W + 1)), int(rng.integers(1, H + 1))
        if k % 3 == 0:
            img = rng.integers(0, 4, size=(H, W, C)).astype(np.uint8)   # many exact ties
        else:
            img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        _carve_cmp(dev, img, tw, th, plain=(k % 2 == 0))


def test_carve_config1(dev):
    job = synth.config1()
    _carve_cmp(dev, job.make(), job.target_w, job.target_h)


def test_carve_generated_multi_cta(dev):
    """A generated image wide enough for a multi-CTA cluster and tall enough for several
    super-tiles, with a ragged last tile; both passes."""
    img = synth.gen_image(700, 333, 12, 20, 200, 91)
    _carve_cmp(dev, img, 650, 300)


@pytest.mark.parametrize("H", [4111, 4112])
def test_carve_tall_heavy_edges(dev, H):
    """Tall carves (4111 and 4112 rows, 64-row super-tiles' ragged ends, seam sums past 2^23)
    with maximum-energy pixels next to both image edges and random ones in between: both equal the
    oracle (seam log, costs, bytes)."""
    yy, xx = np.mgrid[0:H, 0:70]
    img = (((yy + xx) & 1) * 255).astype(np.uint8)[:, :, None].repeat(4, axis=2)   # e1 = 2040 everywhere
    img[:, 30:40] = np.random.default_rng(H).integers(0, 256, size=(H, 10, 4)).astype(np.uint8)
    _carve_cmp(dev, img, 66, H)


@pytest.mark.parametrize("top", [8191, 8192])
def test_find_seam_heavy_edges(dev, top):
    """Caller maps with their largest energy (seam sums on either side of 2^23 at H = 1024) in the
    edge columns and ties everywhere else: seam and cost equal the oracle's, for map widths that end
    inside a lane and on a lane boundary."""
    rng = np.random.default_rng(top)
    for W in (257, 256, 1029, 1920):
        e = rng.integers(0, 3, size=(1024, W)).astype(np.uint16)
        e[:, :3] = top
        e[:, -2:] = top
        e[5, W // 2] = top
        seam, cost = sc.find_seam(_to_dev(e, dev))
        sc.check()
        s_ref, c_ref = oracle.dp_seam(e)
        assert int(_np(cost)[0]) == c_ref, W
        np.testing.assert_array_equal(_np(seam), s_ref, err_msg=f"W={W}")


def test_carve_config2_full(dev):
    """1920x1080 -> 1440 (480 vertical seams): every seam index and every output byte."""
    job = synth.config2()
    _carve_cmp(dev, job.make(), job.target_w, job.target_h)


def test_plain_and_fast_paths_agree(dev):
    img = synth.gen_image(400, 260, 8, 20, 120, 5)
    a = _np(sc.carve(_to_dev(img, dev), 330, 220))
    b = _np(sc.carve(_to_dev(img, dev), 330, 220, plain=True))
    np.testing.assert_array_equal(a, b)


def test_carve_host_entry_point(dev):
    img = synth.gen_image(300, 200, 6, 20, 100, 17)
    out = sc.carve_host(img, 250, 180)
    np.testing.assert_array_equal(out, oracle.carve(img, 250, 180))


def test_batch_equals_alone(dev):
    jobs = synth.config4(n=6, seed=44)
    imgs = [j.make() for j in jobs]
    d = [_to_dev(i, dev) for i in imgs]
    outs, logs = sc.carve_batch(d, [(j.target_w, j.target_h) for j in jobs], with_log=True)
    sc.check()
    for img, j, o, lg in zip(imgs, jobs, outs, logs):
        r_out, r_log, _ = _carve_ref(img, j.target_w, j.target_h)
        np.testing.assert_array_equal(_np(o), r_out)
        np.testing.assert_array_equal(_np(lg)[: len(r_log)], r_log)


def test_invalid_arguments_raise(dev):
    img = _to_dev(np.zeros((10, 10, 3), dtype=np.uint8), dev)
    with pytest.raises(sc.ScError):
        sc.carve(img, 11, 10)
    with pytest.raises(sc.ScError):
        sc.carve(img, 0, 10)


@pytest.mark.slow
def test_carve_config3_full(dev):
    """3840x2160 -> 2880x1620: 960 vertical then 540 horizontal seams (through the transpose), every
    seam index, cost and output byte. The oracle (about a minute of CPU) runs in a thread while the
    GPU carves."""
    import threading
    job = synth.config3()
    img = job.make()
    ref = {}
    th = threading.Thread(target=lambda: ref.update(r=oracle.carve(img, job.target_w, job.target_h, with_log=True)))
    th.start()
    out, log, cost = sc.carve(_to_dev(img, dev), job.target_w, job.target_h, with_log=True)
    sc.check()
    out, log, cost = _np(out), _np(log), _np(cost)
    th.join()
    r_out, r_log, r_cost = ref["r"]
    np.testing.assert_array_equal(log, r_log)
    np.testing.assert_array_equal(cost, r_cost)
    np.testing.assert_array_equal(out, r_out)
