"""The seeded input generator: published splitmix64 values, determinism and the workload shapes."""
import numpy as np

from paper_2410_21207_gb300 import synth


def test_splitmix64_reference_value():
    # splitmix64 seeded with 0: the first output is the published 0xE220A8397B1DCDAF.
    assert int(synth.SplitMix64(0).u64(1)[0]) == 0xE220A8397B1DCDAF


def test_splitmix64_counter_form_matches_sequential():
    def seq(seed, n):
        s, out = seed, []
        for _ in range(n):
            s = (s + 0x9E3779B97F4A7C15) & (2 ** 64 - 1)
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2 ** 64 - 1)
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2 ** 64 - 1)
            out.append(z ^ (z >> 31))
        return out
    r = synth.SplitMix64(12345)
    a = [int(x) for x in r.u64(5)] + [int(x) for x in r.u64(3)]
    assert a == seq(12345, 8)


def test_uniform_and_randint_ranges():
    r = synth.SplitMix64(1)
    u = r.u01(10000)
    assert u.min() >= 0 and u.max() < 1
    k = r.randint(3, 5, 10000)
    assert set(np.unique(k).tolist()) == {3, 4, 5}


def test_generator_deterministic_and_shaped():
    a = synth.gen_image(97, 61, 5, 10, 40, 77)
    b = synth.gen_image(97, 61, 5, 10, 40, 77)
    assert a.shape == (61, 97, 3) and a.dtype == np.uint8
    np.testing.assert_array_equal(a, b)
    c = synth.gen_image(97, 61, 5, 10, 40, 78)
    assert (a != c).any()
    # noise sigma 8 around the flat regions: many distinct values, exact ties still occur
    assert len(np.unique(a)) > 50


def test_configs():
    j1 = synth.config1()
    img = j1.make()
    assert img.shape == (48, 64, 3) and j1.seams == 16
    np.testing.assert_array_equal(img, synth.config1().make())
    assert abs(synth.config2().mpix_seams() - 871.2) < 0.1
    j3 = synth.config3()
    assert j3.W - j3.target_w == 960 and j3.H - j3.target_h == 540
    assert abs(j3.mpix_seams() - 9908.4) < 0.1
    b = synth.config4()
    assert len(b) == 256
    for j in b:
        assert 240 <= j.W <= 1280 and 180 <= j.H <= 960 and j.target_h == j.H
        assert 0.09 * j.W <= j.W - j.target_w <= 0.41 * j.W
    reqs = synth.config5(n=500)
    ts = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(ts) > 0)
    assert 1.5 < ts[-1] < 3.5          # 500 arrivals at 200/s
    for r in reqs:
        assert 128 <= r.W <= 4096 and 128 <= r.H <= 2160
        assert 1 <= r.target_w <= r.W and 1 <= r.target_h <= r.H
