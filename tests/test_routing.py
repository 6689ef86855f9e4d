"""The batched form's scheduler on the host (sc_batch_route, no device call): which images a batch
plan carves on one CTA and which on a cluster, checked against the rules it states."""
import math

import pytest

from paper_2410_21207_gb300 import binding as sc
from paper_2410_21207_gb300 import synth


def _sizes(jobs, C=3):
    return [(j.H, j.W, C, j.target_w, j.target_h) for j in jobs]


def test_balanced_routing_follows_the_share_rule():
    """Images whose estimated one-CTA carve exceeds thr x the mean share per SM go to clusters of
    the 32-row-tile shape with max(2, ceil(W / 384)) CTAs; all others stay on one CTA."""
    jobs = synth.config4()
    sizes = _sizes(jobs)
    for thr in (1.0, 1.4, 2.0):
        cs, shape, us = sc.batch_route(sizes, thr, 152)
        share = sum(us) / 152
        for (H, W, C, tw, th), c, s, u in zip(sizes, cs, shape, us):
            if u > thr * share:
                assert s == 1 and c == max(2, math.ceil(W / 384)), (W, H, c, s)
            else:
                assert c == 0, (W, H, c)
    routed = [c for c in sc.batch_route(sizes, 1.4, 152)[0] if c > 0]
    assert 0 < len(routed) < len(sizes)


def test_no_balancing_keeps_one_cta_images_on_one_cta():
    jobs = synth.config4()
    cs, shape, us = sc.batch_route(_sizes(jobs), 0.0, 152)
    assert all(c == 0 for c in cs)   # every config-4 image fits one CTA (W <= 1280)


def test_wide_images_take_the_8_row_tile_clusters():
    """An image wider than one CTA of the default configuration (1440 columns) goes to clusters of
    the 8-row-tile shape, 768 columns per CTA, whatever the threshold says."""
    sizes = [(100, 2000, 3, 1900, 100), (60, 4000, 1, 3990, 60), (50, 300, 4, 290, 50)]
    cs, shape, us = sc.batch_route(sizes, 0.0, 152)
    assert cs == [3, 6, 0] and shape[:2] == [0, 0]


def test_one_cta_estimate_grows_with_the_work():
    base = (500, 600, 3, 500, 500)
    taller = (900, 600, 3, 500, 900)
    wider = (500, 1000, 3, 900, 500)
    more_seams = (500, 600, 3, 400, 500)
    us = sc.batch_route([base, taller, wider, more_seams], 0.0, 152)[2]
    assert 0 < us[0] < us[1] and us[0] < us[2] and us[0] < us[3]
    # a horizontal pass adds its own seams' time
    both = sc.batch_route([(500, 600, 3, 500, 450)], 0.0, 152)[2][0]
    assert both > us[0]


@pytest.mark.parametrize("sizes,thr,sms", [
    ([], 1.4, 152),
    ([(10, 10, 3, 5, 10)], -1.0, 152),
    ([(10, 10, 3, 5, 10)], 1.4, 0),
    ([(10, 10, 2, 5, 10)], 1.4, 152),    # C must be 1, 3 or 4
    ([(10, 10, 3, 11, 10)], 1.4, 152),   # no enlargement here
])
def test_routing_argument_errors(sizes, thr, sms):
    with pytest.raises(sc.ScError) as ei:
        sc.batch_route(sizes, thr, sms)
    assert ei.value.code == sc.SC_EINVAL
