"""The serving form: requests admitted by a device-memory budget and carved in overlapping
micro-batches / cluster launches; every result equals the same image carved alone."""
import time

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


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        if k % 7 == 3:
            W, H = int(rng.integers(1500, 2300)), int(rng.integers(60, 200))   # wider than one CTA
        else:
            W, H = int(rng.integers(16, 700)), int(rng.integers(8, 400))
        img = synth.gen_image(W, H, 3, 4, 60, 1000 * seed + k)
        tw = max(1, int(W * rng.uniform(0.5, 0.95)))
        th = max(1, int(H * rng.uniform(0.8, 1.0)))
        out.append((img, tw, th))
    return out


def test_served_results_equal_alone(dev):
    reqs = _requests(36, 3)
    srv = sc.Server(budget_bytes=1 << 30, max_batch=8, streams=6)
    tickets = []
    for k, (img, tw, th) in enumerate(reqs):
        tickets.append(srv.submit(img, tw, th, pinned=(k % 3 != 1)))   # some pageable buffers
        if k % 5 == 0:
            time.sleep(0.002)   # later requests arrive while earlier ones are on the GPU
    srv.drain(300)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["device_errors"] == 0
    assert st["batched"] + st["cluster_path"] == len(reqs)
    assert st["cluster_path"] >= 1 and st["groups"] < len(reqs)   # some requests shared a launch
    assert st["peak_bytes"] <= st["budget_bytes"]
    for k, ((img, tw, th), t) in enumerate(zip(reqs, tickets)):
        done, lat = srv.poll(t)
        assert done and lat > 0
        alone = sc.carve(torch.from_numpy(img).to(dev), tw, th).cpu().numpy()
        np.testing.assert_array_equal(srv.result(t), alone)
        if k % 4 == 0 and img.shape[1] < 800:
            np.testing.assert_array_equal(srv.result(t), oracle.carve(img, tw, th))
    srv.close()


def test_admission_waits_for_memory(dev):
    """A budget far smaller than the whole workload: requests wait for memory, none is lost."""
    reqs = _requests(20, 5)
    reqs = [r for r in reqs if r[0].shape[1] < 1400]
    srv = sc.Server(budget_bytes=64 << 20, max_batch=16, streams=4)
    tickets = [srv.submit(img, tw, th) for img, tw, th in reqs]
    srv.drain(300)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["peak_bytes"] <= 64 << 20
    for (img, tw, th), t in zip(reqs, tickets):
        np.testing.assert_array_equal(srv.result(t), oracle.carve(img, tw, th))
    with pytest.raises(sc.ScError):
        srv.submit(np.zeros((4000, 4000, 3), dtype=np.uint8), 3000, 4000)   # larger than the budget
    srv.close()


def test_request_completes_with_its_own_image(dev):
    """Small images batched with a long one complete long before it (per-image completion)."""
    big = synth.gen_image(1300, 900, 3, 6, 200, 71)
    smalls = [synth.gen_image(60 + 7 * k, 40 + 3 * k, 3, 2, 20, 80 + k) for k in range(6)]
    srv = sc.Server(budget_bytes=1 << 30, max_batch=16, streams=2)
    tb = srv.submit(big, 700, 900)
    ts = [srv.submit(im, im.shape[1] - 10, im.shape[0]) for im in smalls]
    srv.drain(300)
    st = srv.stats()
    assert st["completed"] == 7 and st["device_errors"] == 0
    _, lat_big = srv.poll(tb)
    lat_small = [srv.poll(t)[1] for t in ts]
    assert max(lat_small) < 0.5 * lat_big, (lat_small, lat_big)
    np.testing.assert_array_equal(srv.result(tb), oracle.carve(big, 700, 900))
    for im, t in zip(smalls, ts):
        np.testing.assert_array_equal(srv.result(t), oracle.carve(im, im.shape[1] - 10, im.shape[0]))
    srv.close()


def test_heavy_narrow_request_goes_to_a_cluster(dev):
    """A request one CTA covers (600 columns) but whose carve there would take well over 50 ms by the
    carving-time model (2000 rows, 300 seams) is carved by a latency-shaped cluster; a light one
    stays on one CTA. Both equal the oracle's carve."""
    heavy = synth.gen_image(600, 2000, 12, 20, 200, 91)
    light = synth.gen_image(300, 200, 4, 10, 60, 92)
    srv = sc.Server(budget_bytes=1 << 30, max_batch=8, streams=2)
    th_ = srv.submit(heavy, 300, 2000)
    tl = srv.submit(light, 250, 200)
    srv.drain(300)
    st = srv.stats()
    assert st["completed"] == 2 and st["device_errors"] == 0
    assert st["cluster_path"] == 1 and st["batched"] == 1, st
    np.testing.assert_array_equal(srv.result(th_), oracle.carve(heavy, 300, 2000))
    np.testing.assert_array_equal(srv.result(tl), oracle.carve(light, 250, 200))
    srv.close()
