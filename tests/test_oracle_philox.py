"""Pins the oracle's Philox4x32-10 against the published known-answer vectors."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        w = [int(t, 16) for t in lhs.split()]
        o = [int(t, 16) for t in rhs.split()]
        rows.append((w[:4], w[4:], o))
    return rows


def test_known_answer_vectors(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == out


def test_counter_words_all_matter(orc):
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] ^= 1
        assert not np.array_equal(orc.philox4x32_10(c, [5, 6]), base)
    for k in range(2):
        key = [5, 6]
        key[k] ^= 1
        assert not np.array_equal(orc.philox4x32_10([1, 2, 3, 4], key), base)
