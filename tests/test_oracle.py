"""Pins for the oracle: each checks it against something other than itself (hand-worked values,
closed forms, exhaustive enumeration, invariants from the paper, textbook identities)."""
import os

import numpy as np
import pytest

import oracle
from paper_2410_21207_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_cases(name):
    cases = []
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.split("#")[0].strip() for ln in f]
    lines = [ln for ln in lines if ln]
    i = 0
    while i < len(lines):
        hdr = lines[i].split()
        assert hdr[0] == "case"
        cases.append((hdr[1], [int(x) for x in hdr[2:]], []))
        i += 1
        while i < len(lines) and not lines[i].startswith("case"):
            cases[-1][2].append(lines[i])
            i += 1
    return cases


def _energy_cases():
    out = []
    for name, dims, body in _read_cases("energy_examples.txt"):
        H, W, C = dims
        nums = [int(x) for x in " ".join(body).split()]
        assert len(nums) == H * W * C + H * W
        img = np.array(nums[: H * W * C], dtype=np.uint8).reshape(H, W, C)
        e = np.array(nums[H * W * C:], dtype=np.uint16).reshape(H, W)
        out.append((name, img, e))
    return out


def _dp_cases():
    out = []
    for name, dims, body in _read_cases("dp_examples.txt"):
        H, W = dims
        rows = [ln for ln in body if ln[0].isdigit()]
        tags = {ln.split()[0]: [int(x) for x in ln.split()[1:]] for ln in body if not ln[0].isdigit()}
        e = np.array([[int(x) for x in r.split()] for r in rows], dtype=np.uint16)
        assert e.shape == (H, W)
        out.append((name, e, tags))
    return out


@pytest.mark.parametrize("name,img,expected", _energy_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_energy_hand_computed(name, img, expected):
    np.testing.assert_array_equal(oracle.energy(img), expected)


@pytest.mark.parametrize("name,e,tags", _dp_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_dp_hand_worked(name, e, tags):
    seam, cost = oracle.dp_seam(e)
    assert seam.tolist() == tags["seam"]
    assert cost == tags["cost"][0]
    gseam, gcost = oracle.greedy_seam(e)
    assert gseam.tolist() == tags["greedy"][:-1]
    assert gcost == tags["greedy"][-1]
    bseam, bcost, _ = oracle.brute_seam(e)
    assert bseam.tolist() == tags["seam"] and bcost == tags["cost"][0]


def _patterns(rng, H, W):
    yield "uniform", rng.integers(0, 1531, size=(H, W))
    yield "constant", np.full((H, W), int(rng.integers(0, 1531)))
    yield "binary", rng.integers(0, 2, size=(H, W))
    yield "stripes", np.tile(rng.integers(0, 4, size=(1, W)), (H, 1))
    yield "smallrange", rng.integers(0, 4, size=(H, W))


def test_dp_equals_brute_force_tiny():
    """Algorithm 3 finds the same seam (not only the same cost) as exhaustive enumeration of every
    8-connected seam (Algorithm 1) with strict improvement, on every H<=10, W<=12 shape: both
    pick the lexicographically smallest optimal seam read bottom to top."""
    rng = np.random.default_rng(2024)
    n = 0
    for H in range(1, 11):
        for W in range(1, 13):
            if W * 3 ** (H - 1) > 250_000:   # keep the exhaustive search to seconds
                continue
            seeds = 6 if H * W > 40 else 12
            for _ in range(seeds):
                for kind, e in _patterns(rng, H, W):
                    e = e.astype(np.uint16)
                    s1, c1 = oracle.dp_seam(e)
                    s2, c2, _ = oracle.brute_seam(e)
                    assert c1 == c2, (H, W, kind)
                    assert s1.tolist() == s2.tolist(), (H, W, kind, e)
                    n += 1
    assert n > 3000


def test_dp_equals_brute_force_paper_sizes():
    """The brute-force sizes of the runtime experiment (n x n, n = 2, 5, 7, 10; 12 x 12 once)."""
    rng = np.random.default_rng(7)
    for n_, reps in ((2, 40), (5, 40), (7, 20), (10, 3), (12, 1)):
        for _ in range(reps):
            e = rng.integers(0, 6, size=(n_, n_)).astype(np.uint16)
            s1, c1 = oracle.dp_seam(e)
            s2, c2, _ = oracle.brute_seam(e)
            assert c1 == c2 and s1.tolist() == s2.tolist()


def test_brute_force_visits_every_connected_path():
    """The number of 8-connected top-to-bottom paths in an H x W grid is the sum of the entries of
    T^(H-1), T the W x W tridiagonal 0/1 adjacency matrix (walk counting). For H = 1 it is W, and it
    never exceeds the paper's m * 3^(n-1) bound (which ignores the borders)."""
    for H in range(1, 9):
        for W in range(1, 9):
            T = np.eye(W, dtype=np.int64) + np.eye(W, k=1, dtype=np.int64) + np.eye(W, k=-1, dtype=np.int64)
            expect = int(np.linalg.matrix_power(T, H - 1).sum())
            _, _, leaves = oracle.brute_seam(np.zeros((H, W), dtype=np.uint16))
            assert leaves == expect
            assert leaves <= W * 3 ** (H - 1)


def test_brute_force_planted_path():
    """A valid seam of zeros in an image of positive energies is the unique optimum."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        H, W = int(rng.integers(2, 9)), int(rng.integers(2, 10))
        path = [int(rng.integers(0, W))]
        for _ in range(H - 1):
            path.append(int(np.clip(path[-1] + rng.integers(-1, 2), 0, W - 1)))
        e = rng.integers(1, 50, size=(H, W)).astype(np.uint16)
        for i, j in enumerate(path):
            e[i, j] = 0
        for fn in (oracle.dp_seam, oracle.brute_seam):
            r = fn(e)
            assert r[1] == 0 and r[0].tolist() == path


def _valid_seam(seam, H, W):
    assert seam.shape == (H,)
    assert seam.min() >= 0 and seam.max() < W
    assert np.all(np.abs(np.diff(seam)) <= 1)


def test_seam_invariants_and_greedy_bound():
    """One pixel per row, |delta col| <= 1 (Seam Identification); cost = sum of e along the seam;
    DP cost <= greedy cost (greedy is not guaranteed optimal); the DP cost is min of the last row
    of M."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        H, W = int(rng.integers(1, 40)), int(rng.integers(1, 60))
        e = rng.integers(0, 1531, size=(H, W)).astype(np.uint16)
        s, c = oracle.dp_seam(e)
        _valid_seam(s, H, W)
        assert c == int(e[np.arange(H), s].astype(np.int64).sum())
        gs, gc = oracle.greedy_seam(e)
        _valid_seam(gs, H, W)
        assert gc == int(e[np.arange(H), gs].astype(np.int64).sum())
        assert c <= gc
        last = oracle.dp_last_row(e)
        assert c == last.min() and s[-1] == int(np.argmin(last))


def _brute_last_row(e):
    """For every bottom column j, the minimum energy over all 8-connected top-to-bottom paths that
    end at (H-1, j), by enumerating the paths (no recurrence)."""
    H, W = e.shape
    best = [None] * W

    def walk(i, j, acc):   # extend a path that has reached (i, j) with energy acc
        acc += int(e[i, j])
        if i == H - 1:
            if best[j] is None or acc < best[j]:
                best[j] = acc
            return
        for nj in (j - 1, j, j + 1):
            if 0 <= nj < W:
                walk(i + 1, nj, acc)

    for j0 in range(W):
        walk(0, j0, 0)
    return np.array(best, dtype=np.int64)


def test_dp_last_row_is_the_per_column_path_minimum():
    """Every entry of M's last row (Algorithm 3's table, not only its minimum) is the least energy
    of a path ending at that column; this catches a wrong exclusion at either edge or a wrong
    neighbour at any column, minimal or not."""
    rng = np.random.default_rng(163)
    shapes = [(H, W) for H in range(1, 8) for W in range(1, 7)]
    for H, W in shapes:
        for kind in range(3):
            hi = (1531, 3, 65536)[kind]
            e = rng.integers(0, hi, size=(H, W)).astype(np.uint16)
            np.testing.assert_array_equal(oracle.dp_last_row(e), _brute_last_row(e), err_msg=f"{H}x{W} {kind}")
    # edges that must be excluded, not wrapped: a cheap column at the far side of the map would
    # leak into the first or last column through a wrap-around
    e = np.array([[9, 9, 9, 0], [9, 9, 9, 9], [9, 9, 9, 9]], dtype=np.uint16)
    np.testing.assert_array_equal(oracle.dp_last_row(e), _brute_last_row(e))
    assert list(oracle.dp_last_row(e)) == [27, 18, 18, 18]   # by hand: row 1 is [18, 18, 9, 9]; a wrap would give 18 at column 0


def test_closed_forms():
    rng = np.random.default_rng(9)
    # constant image: zero energy, the leftmost straight seam
    img = np.full((13, 17, 3), 77, dtype=np.uint8)
    assert not oracle.energy(img).any()
    s, c = oracle.dp_seam(oracle.energy(img))
    assert c == 0 and not s.any()
    # column-only energy: the straight seam at the leftmost column of minimal energy, cost H*min
    for _ in range(50):
        H, W = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        col = rng.integers(0, 20, size=W)
        e = np.tile(col, (H, 1)).astype(np.uint16)
        s, c = oracle.dp_seam(e)
        j = int(np.argmin(col))
        assert s.tolist() == [j] * H and c == H * int(col[j])
    # H = 1: the textbook leftmost argmin
    for _ in range(50):
        W = int(rng.integers(1, 50))
        e = rng.integers(0, 5, size=(1, W)).astype(np.uint16)
        s, c = oracle.dp_seam(e)
        assert s[0] == int(np.argmin(e[0])) and c == int(e[0].min())


def test_energy_properties():
    rng = np.random.default_rng(3)
    for _ in range(40):
        H, W, C = int(rng.integers(1, 20)), int(rng.integers(1, 20)), int(rng.choice([1, 3, 4]))
        img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        e = oracle.energy(img)
        # the formula is symmetric in rows and columns: e(I^T) = e(I)^T
        np.testing.assert_array_equal(oracle.energy(img.transpose(1, 0, 2)), e.T)
        # channels add
        parts = sum(oracle.energy(img[:, :, c:c + 1]).astype(np.int64) for c in range(C))
        np.testing.assert_array_equal(parts, e)
        assert e.max() <= 2 * 255 * C
    # a horizontal ramp I(i,j) = a*j: x term 2a inside, a at the two border columns; y term 0
    for a in (1, 3, 7):
        W = 9
        img = np.tile((a * np.arange(W, dtype=np.uint8))[None, :, None], (4, 1, 1))
        e = oracle.energy(img)
        expect = np.full(W, 2 * a)
        expect[0] = expect[-1] = a
        np.testing.assert_array_equal(e, np.tile(expect, (4, 1)))
    # one column: the x term vanishes (both neighbours clamp to the pixel)
    img = rng.integers(0, 256, size=(6, 1, 3)).astype(np.uint8)
    e = oracle.energy(img)
    dy = np.abs(img[np.minimum(np.arange(6) + 1, 5)].astype(int) - img[np.maximum(np.arange(6) - 1, 0)].astype(int))
    np.testing.assert_array_equal(e[:, 0], dy.sum(axis=2)[:, 0])


def test_remove_seam():
    """Every output row is its input row with exactly the seam pixel deleted, order kept."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        H, W, C = int(rng.integers(1, 10)), int(rng.integers(2, 12)), 3
        img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        seam = np.array([int(rng.integers(0, W)) for _ in range(H)], dtype=np.int32)
        out = oracle.remove_seam(img, seam)
        for i in range(H):
            np.testing.assert_array_equal(out[i], np.delete(img[i], seam[i], axis=0))


def test_local_refresh_dirty_set():
    """After removing a seam s (|s_i - s_(i-1)| <= 1), the full energy recompute equals the
    energy shifted left past s everywhere except the new columns s_i - 1 and s_i of each row."""
    rng = np.random.default_rng(6)
    for _ in range(200):
        H, W = int(rng.integers(1, 14)), int(rng.integers(2, 16))
        img = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
        e = oracle.energy(img)
        s, _ = oracle.dp_seam(e)
        if rng.random() < 0.5:   # any connected seam, not only the optimum
            s = [int(rng.integers(0, W))]
            for _ in range(H - 1):
                s.append(int(np.clip(s[-1] + rng.integers(-1, 2), 0, W - 1)))
            s = np.array(s, dtype=np.int32)
        e2 = oracle.energy(oracle.remove_seam(img, s))
        for i in range(H):
            shifted = np.delete(e[i], s[i])
            dirty = {s[i] - 1, s[i]}
            for j in range(W - 1):
                if j not in dirty:
                    assert e2[i, j] == shifted[j], (i, j)


def test_carve_invariants():
    rng = np.random.default_rng(8)
    for _ in range(20):
        H, W = int(rng.integers(2, 20)), int(rng.integers(2, 20))
        tw, th = int(rng.integers(1, W + 1)), int(rng.integers(1, H + 1))
        img = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
        out, log, costs = oracle.carve(img, tw, th, with_log=True)
        assert out.shape == (th, tw, 3)
        nv = W - tw
        # every vertical seam is valid in the image it was found in, and mapping the log back to
        # original columns deletes each original pixel at most once
        cols = np.tile(np.arange(W), (H, 1))
        removed = np.zeros((H, W), dtype=np.int64)
        for t in range(nv):
            s = log[t * H:(t + 1) * H]
            _valid_seam(s, H, W - t)
            for i in range(H):
                removed[i, cols[i, s[i]]] += 1
                cols[i] = np.concatenate([np.delete(cols[i, :W - t], s[i]), [-1] * (t + 1)])
        assert removed.max() <= 1 and removed.sum() == nv * H
        if th == H:
            # with only vertical seams, the output keeps exactly the surviving original pixels
            for i in range(H):
                keep = np.nonzero(removed[i] == 0)[0]
                np.testing.assert_array_equal(out[i], img[i, keep])


def test_constant_image_carve():
    img = np.full((9, 12, 3), 200, dtype=np.uint8)
    out, log, costs = oracle.carve(img, 7, 6, with_log=True)
    assert (out == 200).all() and out.shape == (6, 7, 3)
    assert not log.any() and not costs.any()   # every seam is the leftmost straight one, cost 0


def test_horizontal_pass_is_transposed_vertical():
    """Horizontal seams are vertical seams of the transposed image ('Design Techniques'): carving
    H -> th equals transpose, remove H - th vertical seams, transpose back."""
    rng = np.random.default_rng(10)
    for _ in range(10):
        H, W = int(rng.integers(3, 16)), int(rng.integers(3, 16))
        tw, th = int(rng.integers(1, W + 1)), int(rng.integers(1, H + 1))
        img = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
        out = oracle.carve(img, tw, th)
        stage1 = oracle.carve(img, tw, H)
        via_t = oracle.carve(oracle.transpose(stage1), th, tw)
        np.testing.assert_array_equal(out, oracle.transpose(via_t))
        np.testing.assert_array_equal(oracle.transpose(oracle.transpose(img)), img)


def test_config1_oracle_small():
    """Config 1 (64x48, 16 seams) runs through the oracle; its seams are valid and crops of its
    first energy map agree with brute force."""
    job = synth.config1()
    img = job.make()
    out, log, costs = oracle.carve(img, job.target_w, job.target_h, with_log=True)
    assert out.shape == (48, 48, 3)
    e = oracle.energy(img)
    for t in range(16):
        _valid_seam(log[t * 48:(t + 1) * 48], 48, 64 - t)
    rng = np.random.default_rng(1)
    for _ in range(5):
        i0, j0 = int(rng.integers(0, 48 - 10)), int(rng.integers(0, 64 - 12))
        crop = e[i0:i0 + 10, j0:j0 + 12]
        s1, c1 = oracle.dp_seam(crop)
        s2, c2, _ = oracle.brute_seam(crop)
        assert c1 == c2 and s1.tolist() == s2.tolist()


# ---- seam insertion (reading R9) ----

def _enlarge_cases():
    rng = np.random.default_rng(917)
    cases = []
    for H, W, C in [(1, 2, 1), (1, 9, 3), (3, 2, 3), (4, 5, 1), (7, 12, 4), (16, 23, 3), (33, 40, 3), (50, 9, 1)]:
        for kind in ("uniform", "ties"):
            hi = 256 if kind == "uniform" else 3
            img = rng.integers(0, hi, size=(H, W, C)).astype(np.uint8)
            for k in sorted({1, max(1, W // 3), W - 1}):
                cases.append((img, k))
    return cases


def test_enlarge_deleting_the_inserted_pixels_gives_the_input():
    """Each row holds exactly k inserted pixels, right after k distinct input columns, with the
    rounded-up mean of that pixel and its right neighbour; deleting them restores the row."""
    for img, k in _enlarge_cases():
        H, W, C = img.shape
        out, cols = oracle.enlarge(img, W + k, with_cols=True)
        assert out.shape == (H, W + k, C) and cols.shape == (k, H)
        for i in range(H):
            d = np.sort(cols[:, i])
            assert len(set(d.tolist())) == k and d.min() >= 0 and d.max() < W
            ins = d + np.arange(k) + 1                    # output positions of the inserted pixels
            keep = np.setdiff1d(np.arange(W + k), ins)
            np.testing.assert_array_equal(out[i, keep], img[i])
            right = img[i, np.minimum(d + 1, W - 1)].astype(np.int32)
            mean = (img[i, d].astype(np.int32) + right + 1) // 2
            np.testing.assert_array_equal(out[i, ins], mean.astype(np.uint8))


def test_enlarge_columns_are_the_carved_seams():
    """The k mapped columns of a row are exactly the pixels the carve to W - k deletes from it."""
    for img, k in _enlarge_cases():
        H, W, C = img.shape
        _, cols = oracle.enlarge(img, W + k, with_cols=True)
        carved = oracle.carve(img, W - k, H)
        for i in range(H):
            keep = np.setdiff1d(np.arange(W), cols[:, i])
            np.testing.assert_array_equal(img[i, keep], carved[i])


def test_enlarge_constant_image_and_limits():
    img = np.full((6, 10, 3), 77, dtype=np.uint8)
    np.testing.assert_array_equal(oracle.enlarge(img, 19), np.full((6, 19, 3), 77, dtype=np.uint8))
    for tw in (10, 20, 5):
        with pytest.raises(ValueError):
            oracle.enlarge(img, tw)


# ---- forward energy (reading R10) ----

def _new_pair_cost(img, seam):
    """Sum of the L1 colour differences of the pixel pairs that are adjacent in the image with
    `seam` removed but were not adjacent before: computed from the two images alone."""
    H, W, C = img.shape
    src = [[j for j in range(W) if j != seam[i]] for i in range(H)]   # input column of each output pixel
    tot = 0
    img = img.astype(np.int64)

    def diff(a, b):
        return int(np.abs(img[a] - img[b]).sum())

    for i in range(H):
        for jj in range(W - 1):
            if jj + 1 < W - 1:
                a, b = (i, src[i][jj]), (i, src[i][jj + 1])
                if abs(a[1] - b[1]) != 1:
                    tot += diff(a, b)
            if i + 1 < H:
                a, b = (i, src[i][jj]), (i + 1, src[i + 1][jj])
                if a[1] != b[1]:
                    tot += diff(a, b)
    return tot


def _all_seams(H, W):
    """Every 8-connected seam, bottom column ascending, each step up col-1, col, col+1."""
    def up(i, col, path):
        if i < 0:
            yield list(reversed(path))
            return
        for c in (col - 1, col, col + 1):
            if 0 <= c < W:
                yield from up(i - 1, c, path + [c])
    for col in range(W):
        yield from up(H - 2, col, [col])


def _path_cost(planes, seam):
    cu, dl, dr = planes
    c = int(cu[0, seam[0]])
    for i in range(1, len(seam)):
        j, jp = seam[i], seam[i - 1]
        c += int(cu[i, j]) + (int(dl[i, j]) if jp == j - 1 else 0) + (int(dr[i, j]) if jp == j + 1 else 0)
    return c


def test_forward_costs_are_the_new_adjacencies():
    """Along any seam, the forward costs add up to the colour differences of the pairs its removal
    makes adjacent (borders included): the planes are pinned to what forward energy means."""
    rng = np.random.default_rng(2008)
    for H, W, C in [(1, 2, 1), (1, 5, 3), (2, 2, 3), (3, 4, 1), (4, 5, 3), (5, 6, 4), (6, 3, 3)]:
        for _ in range(4):
            img = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
            planes = oracle.forward_costs(img)
            seams = list(_all_seams(H, W))
            for s in seams[:: max(1, len(seams) // 40)]:
                assert _path_cost(planes, s) == _new_pair_cost(img, s), (H, W, C, s)


def test_forward_dp_equals_brute_force():
    """The forward DP seam is the first strictly cheapest seam of the exhaustive enumeration (the
    lexicographically smallest optimal seam read bottom to top), cost included."""
    rng = np.random.default_rng(2009)
    for H, W in [(1, 1), (1, 6), (2, 3), (3, 3), (4, 5), (5, 6), (6, 4), (3, 8)]:
        for kind in ("uniform", "ties"):
            for _ in range(6):
                hi = 256 if kind == "uniform" else 2
                img = rng.integers(0, hi, size=(H, W, 3)).astype(np.uint8)
                planes = oracle.forward_costs(img)
                best, best_s = None, None
                for s in _all_seams(H, W):
                    c = _path_cost(planes, s)
                    if best is None or c < best:
                        best, best_s = c, s
                seam, cost = oracle.dp_seam_forward(*planes)
                assert cost == best, (H, W, kind)
                np.testing.assert_array_equal(seam, best_s)


def test_forward_carve_invariants():
    img = np.full((7, 9, 3), 40, dtype=np.uint8)
    np.testing.assert_array_equal(oracle.carve_forward(img, 5, 4), np.full((4, 5, 3), 40, dtype=np.uint8))
    rng = np.random.default_rng(2010)
    img = rng.integers(0, 256, size=(12, 15, 3)).astype(np.uint8)
    out, log, costs = oracle.carve_forward(img, 10, 12, with_log=True)
    cur = img
    for t in range(5):
        s = log[t * 12:(t + 1) * 12]
        assert costs[t] == _new_pair_cost(cur, s)   # each removal's cost is what it makes adjacent
        cur = oracle.remove_seam(cur, s)
    np.testing.assert_array_equal(out, cur)
    # horizontal seams are the vertical seams of the transposed image
    t_out = oracle.carve_forward(img.transpose(1, 0, 2).copy(), 10, 15)
    np.testing.assert_array_equal(oracle.carve_forward(img, 15, 10), t_out.transpose(1, 0, 2))
