"""The batched persistent form (sc_carve_batch, batch plans): every image equals the oracle's carve
of that image alone, byte for byte, including the seam log."""
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


def _mixed_batch(rng):
    imgs, targets = [], []
    shapes = [(1, 1, 3), (2, 3, 1), (5, 40, 4), (40, 7, 3), (61, 97, 3), (180, 240, 3), (33, 1000, 3),
              (300, 700, 1), (100, 1500, 3), (70, 2000, 3), (1500, 90, 3)]
    for H, W, C in shapes:
        if rng.random() < 0.3:
            img = rng.integers(0, 3, size=(H, W, C)).astype(np.uint8)      # many exact ties
        else:
            img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        tw = int(rng.integers(max(1, W // 2), W + 1))
        th = int(rng.integers(max(1, (3 * H) // 4), H + 1))
        imgs.append(img)
        targets.append((tw, th))
    return imgs, targets


def _check(imgs, targets, outs, logs):
    for img, (tw, th), o, lg in zip(imgs, targets, outs, logs):
        r_out, r_log, _ = oracle.carve(img, tw, th, with_log=True)
        np.testing.assert_array_equal(o.cpu().numpy().reshape(r_out.shape), r_out)
        np.testing.assert_array_equal(lg.cpu().numpy()[: len(r_log)], r_log)


def test_batch_mixed_sizes_equal_alone(dev):
    """Sizes from 1x1 to 2000 wide, both passes, C in {1,3,4}; the widest go to the cluster path."""
    rng = np.random.default_rng(404)
    imgs, targets = _mixed_batch(rng)
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    outs, logs = sc.carve_batch(d, targets, with_log=True)
    sc.check()
    _check(imgs, targets, outs, logs)


def test_batch_config4_subset_equal_alone(dev):
    jobs = synth.config4(n=24, seed=4)
    imgs = [j.make() for j in jobs]
    targets = [(j.target_w, j.target_h) for j in jobs]
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    outs, logs = sc.carve_batch(d, targets, with_log=True)
    sc.check()
    _check(imgs, targets, outs, logs)


def test_batch_plan_autotuned_replays(dev):
    """An autotuned plan (CUDA graph) replays correctly, also after the inputs change in place."""
    rng = np.random.default_rng(9)
    imgs = [synth.gen_image(int(rng.integers(60, 500)), int(rng.integers(40, 300)), 5, 10, 80, 100 + k)
            for k in range(10)]
    targets = [(max(1, (4 * im.shape[1]) // 5), im.shape[0] - (k % 3) * 5) for k, im in enumerate(imgs)]
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    plan = sc.BatchPlan(d, targets, autotune=True, with_log=True)
    info = plan.info()
    # with idle SMs the autotuner may carve some images on latency-shaped clusters instead
    assert info["batched"] + info["cluster_path"] == len(imgs)
    assert info["tile_rows"] in (8, 16, 32)
    for rep in range(2):
        plan.run()
        sc.check()
        _check(imgs, targets, plan.outs, plan.logs)
        # new contents, same sizes
        imgs = [synth.gen_image(im.shape[1], im.shape[0], 5, 10, 80, 500 + rep * 10 + k) for k, im in enumerate(imgs)]
        for t, im in zip(d, imgs):
            t.copy_(torch.from_numpy(im))
    plan.close()


def _wide_batch(rng):
    """Images wider than any one-CTA configuration (cluster sizes 3 to 6 of the cluster kernel), a
    tall one whose horizontal pass is the wide search, and two small ones in the same batch."""
    shapes = [(64, 1800, 3, 40, 0), (40, 2600, 1, 30, 3), (90, 3300, 4, 25, 0), (120, 4096, 3, 20, 6),
              (1700, 50, 3, 4, 30), (33, 200, 3, 10, 2), (70, 2100, 3, 35, 0), (16, 300, 1, 5, 0)]
    imgs, targets = [], []
    for k, (H, W, C, nv, nh) in enumerate(shapes):
        if k % 3 == 1:
            img = rng.integers(0, 3, size=(H, W, C)).astype(np.uint8)      # many exact ties
        else:
            img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        imgs.append(img)
        targets.append((W - nv, H - nh))
    return imgs, targets


def test_batch_wide_images_cluster_kernel(dev):
    rng = np.random.default_rng(77)
    imgs, targets = _wide_batch(rng)
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    outs, logs = sc.carve_batch(d, targets, with_log=True)
    sc.check()
    _check(imgs, targets, outs, logs)


def test_batch_plan_with_wide_images_replays(dev):
    """A plan whose graph holds the one-CTA launch and the cluster launches replays exactly."""
    rng = np.random.default_rng(78)
    imgs, targets = _wide_batch(rng)
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    plan = sc.BatchPlan(d, targets, autotune=False, with_log=True)
    info = plan.info()
    assert info["batched"] + info["cluster_path"] == len(imgs) and info["cluster_path"] >= 5
    for _ in range(2):
        plan.run()
        sc.check()
        _check(imgs, targets, plan.outs, plan.logs)
    plan.close()


def test_balanced_plan_runs_clusters_beside_one_cta_kernel(dev):
    """A batch dominated by one large image: with load balancing (autotune = 2) the large image is
    carved by a cluster of the 32-row-tile shape (1000 columns: 3 CTAs) launched beside the one-CTA
    kernel that carves the small ones (two graph branches); every image still equals the oracle's
    carve of it alone, on two replays."""
    big = synth.gen_image(1000, 700, 8, 20, 200, 2024)
    smalls = [synth.gen_image(120 + 9 * k, 90 + 5 * k, 3, 10, 40, 300 + k) for k in range(24)]
    imgs = [big] + smalls
    targets = [(700, 700)] + [(im.shape[1] - 8 - k % 5, im.shape[0]) for k, im in enumerate(smalls)]
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    plan = sc.BatchPlan(d, targets, autotune=2, with_log=True)
    info = plan.info()
    assert info["cluster_path"] == 1 and info["batched"] == len(smalls)
    for _ in range(2):
        plan.run()
        sc.check()
        _check(imgs, targets, plan.outs, plan.logs)
    plan.close()


def test_balanced_plan_several_cluster_groups(dev):
    """Three cluster groups chained ahead of the one-CTA kernel: two heavy images of
    different widths on 32-row-tile clusters (1000 columns: 3 CTAs, 600 columns: 2 CTAs), one image
    wider than a CTA (1700 columns) on the 8-row-tile shape, and small images on one CTA each; two
    passes for one heavy image. Every image equals the oracle's carve of it alone, on two replays."""
    imgs = [synth.gen_image(1000, 420, 8, 20, 200, 3031), synth.gen_image(600, 500, 6, 20, 150, 3032),
            synth.gen_image(1700, 24, 4, 5, 20, 3033)]
    targets = [(760, 420), (420, 460), (1696, 24)]
    for k in range(20):
        im = synth.gen_image(100 + 7 * k, 80 + 3 * k, 3, 10, 40, 3100 + k)
        imgs.append(im)
        targets.append((im.shape[1] - 5 - k % 4, im.shape[0]))
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    plan = sc.BatchPlan(d, targets, autotune=2, with_log=True)
    info = plan.info()
    assert info["cluster_path"] == 3 and info["batched"] == 20
    for _ in range(2):
        plan.run()
        sc.check()
        _check(imgs, targets, plan.outs, plan.logs)
    plan.close()


def test_route_query_matches_the_balanced_plan(dev):
    """sc_batch_route (host only) predicts the plan's routing: a balanced plan (autotune = 2, the
    1.4 threshold) of the first 96 config-4 images carves on clusters exactly as many images as the
    query sends to clusters for this device's SM count, and every image still equals the oracle."""
    jobs = synth.config4()[:96]
    imgs = [j.make() for j in jobs]
    targets = [(j.target_w, j.target_h) for j in jobs]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cs, shape, us = sc.batch_route([(j.H, j.W, 3, j.target_w, j.target_h) for j in jobs], 1.4, sms)
    routed = sum(1 for c in cs if c > 0)
    assert routed > 0
    d = [torch.from_numpy(i).to(dev) for i in imgs]
    plan = sc.BatchPlan(d, targets, autotune=2, with_log=True)
    info = plan.info()
    assert info["cluster_path"] == routed and info["batched"] == len(jobs) - routed, (info, routed)
    plan.run()
    sc.check()
    for k in range(0, len(jobs), 12):   # a sample against the oracle (the whole batch is in the full-size test)
        _check([imgs[k]], [targets[k]], [plan.outs[k]], [plan.logs[k]])
    plan.close()
