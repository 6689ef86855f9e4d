"""Parity at the sizes and in the launch configurations the benchmark times, element by element
against the oracle: forward energy and seam insertion on the 1920x1080 image, the whole 256-image
batch through an autotuned batch plan, and served requests of the 10,000-request trace up to its
widest, tallest and largest images. The oracle runs in host threads (its C calls release the
GIL) while the GPU works; these tests take minutes and are marked slow."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2410_21207_gb300 import binding as sc
from paper_2410_21207_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    return torch.device("cuda:0")


def _pool():
    return ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2))


def test_forward_carve_1920x1080_full(dev):
    """1920x1080 -> 1440x1080 with forward energy (480 seams): every seam index, cost and byte."""
    job = synth.config2()
    img = job.make()
    with _pool() as ex:
        ref = ex.submit(oracle.carve_forward, img, job.target_w, job.target_h, True)
        out, log, cost = sc.carve_forward(torch.from_numpy(img).to(dev), job.target_w, job.target_h, with_log=True)
        sc.check()
        r_out, r_log, r_cost = ref.result()
    np.testing.assert_array_equal(log.cpu().numpy(), r_log)
    np.testing.assert_array_equal(cost.cpu().numpy(), r_cost)
    np.testing.assert_array_equal(out.cpu().numpy(), r_out)


def test_enlarge_1920_to_2400_full(dev):
    """Seam insertion 1920 -> 2400 (480 seams) on the 1920x1080 image: the inserted columns and
    every output byte."""
    img = synth.config2().make()
    with _pool() as ex:
        ref = ex.submit(oracle.enlarge, img, 2400, True)
        out, cols = sc.enlarge(torch.from_numpy(img).to(dev), 2400, with_cols=True)
        sc.check()
        r_out, r_cols = ref.result()
    np.testing.assert_array_equal(cols.cpu().numpy()[:480], r_cols)
    np.testing.assert_array_equal(out.cpu().numpy(), r_out)


def test_batch_config4_full_autotuned_plan(dev):
    """All 256 images of the batched workload through an autotuned batch plan (the persistent
    launches in a CUDA graph, as the benchmark runs them), replayed twice: every output byte and
    seam log equals the oracle's carve of that image alone."""
    jobs = synth.config4()
    with _pool() as ex:
        imgs = list(ex.map(lambda j: j.make(), jobs))
        refs = [ex.submit(oracle.carve, img, j.target_w, j.target_h, True) for img, j in zip(imgs, jobs)]
        d = [torch.from_numpy(i).to(dev) for i in imgs]
        targets = [(j.target_w, j.target_h) for j in jobs]
        plan = sc.BatchPlan(d, targets, autotune=True, with_log=True)
        info = plan.info()
        assert info["batched"] + info["cluster_path"] == len(jobs)
        for _ in range(2):
            plan.run()
            sc.check()
            for k, (r, o, lg) in enumerate(zip(refs, plan.outs, plan.logs)):
                r_out, r_log, _ = r.result()
                np.testing.assert_array_equal(o.cpu().numpy(), r_out, err_msg=f"image {k} {jobs[k].name}")
                np.testing.assert_array_equal(lg.cpu().numpy()[: len(r_log)], r_log, err_msg=f"image {k}")
        plan.close()


def _trace_subset():
    """Requests of the first 300 of the trace: the three widest, the three tallest, the three
    largest by carving work, and every 20th one."""
    reqs = synth.config5(n=300)
    pick = set()
    pick.update(sorted(range(300), key=lambda k: -reqs[k].W)[:3])
    pick.update(sorted(range(300), key=lambda k: -reqs[k].H)[:3])
    pick.update(sorted(range(300), key=lambda k: -reqs[k].mpix_seams())[:3])
    pick.update(range(0, 300, 20))
    return [reqs[k] for k in sorted(pick)]


def test_served_trace_requests_equal_oracle(dev):
    """At least 20 requests of the serving trace (sizes up to 3830 wide, 2097 tall, the heaviest
    3181x1686 -> 1668x1481) submitted at once to a server with the benchmark's settings: every
    served image equals the oracle's carve byte for byte."""
    reqs = _trace_subset()
    assert len(reqs) >= 20
    with _pool() as ex:
        imgs = list(ex.map(lambda r: r.make(), reqs))
        refs = [ex.submit(oracle.carve, img, r.target_w, r.target_h) for img, r in zip(imgs, reqs)]
        srv = sc.Server(budget_bytes=40 << 30, max_batch=64, streams=16)
        tickets = [srv.submit(img, r.target_w, r.target_h) for img, r in zip(imgs, reqs)]
        srv.drain(900)
        st = srv.stats()
        assert st["completed"] >= len(reqs) and st["device_errors"] == 0
        assert st["cluster_path"] >= 1 and st["batched"] >= 1
        for r, t, ref in zip(reqs, tickets, refs):
            done, _ = srv.poll(t)
            assert done
            np.testing.assert_array_equal(srv.result(t), ref.result(), err_msg=r.name)
        srv.close()
