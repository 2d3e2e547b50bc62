"""Pins the oracle's Morton quantisation on hand-computed points (Sec. III-B,
"Division of the simulation domain": cells indexed along the Morton curve)."""
import numpy as np


def codes(orc, pts, lo=None, hi=None):
    p = np.asarray(pts, np.float32)
    c, l, h = orc.morton(p[:, 0], p[:, 1], p[:, 2], lo, hi)
    return [int(v) for v in c], l, h


def test_unit_box_hand_values(orc):
    lo, hi = [0, 0, 0], [1, 1, 1]
    pts = [(0, 0, 0), (1, 1, 1), (0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5),
           (2.0 ** -10, 0, 0), (0, 2.0 ** -10, 0), (0, 0, 3 * 2.0 ** -10), (0.75, 0, 0)]
    got, _, _ = codes(orc, pts, lo, hi)
    assert got == [0, (1 << 30) - 1, 1 << 27, 1 << 28, 1 << 29, 1, 2, (1 << 2) | (1 << 5),
                   (1 << 27) | (1 << 24)]


def test_offset_box_and_clamping(orc):
    lo, hi = [-1, -1, -1], [1, 1, 1]
    pts = [(0, 0, 0), (-5, -5, -5), (5, 5, 5), (float("nan"), -1, -1)]
    got, _, _ = codes(orc, pts, lo, hi)
    # (0 - -1) * 0.5 * 1024 = 512 on each axis -> bit 9 of x, y, z
    assert got[0] == (1 << 27) | (1 << 28) | (1 << 29)
    assert got[1] == 0                 # below the box clamps to cell 0
    assert got[2] == (1 << 30) - 1     # above the box clamps to cell 1023
    assert got[3] == 0                 # NaN quantises to 0


def test_bounding_box_domain(orc):
    pts = [(10, 20, 30), (14, 28, 31), (12, 24, 30.5)]
    got, lo, hi = codes(orc, pts)
    assert list(lo) == [10, 20, 30] and list(hi) == [14, 28, 31]
    assert got[0] == 0
    assert got[1] == (1 << 30) - 1
    # midpoint on every axis: q = 512 on each axis
    assert got[2] == (1 << 27) | (1 << 28) | (1 << 29)


def test_degenerate_axis(orc):
    pts = [(0, 5, 0), (1, 5, 0)]
    got, lo, hi = codes(orc, pts)
    assert hi[1] == lo[1] == 5
    # x spans the box (q = 1023 on x); y and z collapse to cell 0
    assert got == [0, sum(1 << (3 * b) for b in range(10))]


def test_matches_float32_formula_elementwise(orc):
    # The quantisation is an integer decided in FP32: every single-rounded step
    # is reproduced with numpy float32 scalars, independently of the C code.
    rng = np.random.default_rng(0)
    p = (rng.random((2000, 3)) * 777.0 + 3.0).astype(np.float32)
    got, lo, hi = orc.morton(p[:, 0], p[:, 1], p[:, 2])
    for k in range(0, 2000, 97):
        q = []
        for a in range(3):
            ext = np.float32(hi[a]) - np.float32(lo[a])
            inv = np.float32(1.0) / ext
            t = ((p[k, a] - lo[a]) * inv) * np.float32(1024.0)
            q.append(int(min(max(np.floor(t), 0), 1023)))
        code = 0
        for b in range(10):
            for a in range(3):
                code |= ((q[a] >> b) & 1) << (3 * b + a)
        assert code == int(got[k])
