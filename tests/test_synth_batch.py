"""The mixed-size batch's seeded shapes: deterministic, inside the stated ranges, and
accepted by the library's shape rules (image sides 2^k or 3 * 2^m multiples of 16, at
most n/16 facets a side, nuclear facets with at least L pixels)."""
from __future__ import annotations

import math

import fhs_synth as fs


def test_batch_specs_deterministic_and_in_range():
    a, b = fs.batch_specs(), fs.batch_specs()
    assert [s.name for s in a] == [s.name for s in b]
    assert len(a) == 16
    assert max(s.n for s in a) == 768 and {s.n for s in a} <= set(fs.BATCH_SIDES)
    assert any(s.n % 3 == 0 for s in a) and any(s.n % 3 for s in a)
    for s in a:
        assert 8 <= s.L <= 48 and 1 <= s.Q <= 6 and 0.3 <= s.m_ratio <= 2.0 and 1 <= s.B <= 4
        m = s.n
        while m % 3 == 0:
            m //= 3
        assert m & (m - 1) == 0 and s.n % 16 == 0 and s.n <= 1536
        assert s.Q <= s.n // 16
        t = s.n // s.Q
        side = t + int(math.floor(s.overlap * t))
        assert t * t >= s.L and side * side >= s.L
    assert len({s.seed for s in a}) == 16
    assert [s.name for s in fs.batch_specs(seed=3001)] != [s.name for s in a]
