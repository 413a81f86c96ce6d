"""The accumulation kernels generate the scan phase factor E[v, s] = exp(-2 pi i (v_y s_y / S_y +
v_x s_x / S_x)) (the 2-D scan DFT of Eq. 14) from an exact integer index
    m(s) = ((v_y s_y mod S_y) m_y + (v_x s_x mod S_x) m_x) mod lcm,   m_y = lcm / S_y, m_x = lcm / S_x,
into a table exp(-2 pi i m / lcm).  Between two 16-frame groups 64 scan positions apart they step
the index instead of recomputing it: + 64 v_x m_x along one scan row, and + 64 v_x m_x + v_y m_y
when the 64 positions wrap into the next row (raster order).  These tests restate that rule and
check it, in exact integers, against the index computed from scratch and against the phase
itself, over every frequency of several scan shapes (square, non-square, narrower than 64)."""
import math

import numpy as np
import pytest


def full_index(s, vy, vx, Sy, Sx, lcm):
    sy, sx = divmod(s, Sx)
    return ((vy * sy % Sy) * (lcm // Sy) + (vx * sx % Sx) * (lcm // Sx)) % lcm


def stepped_index(m0, g0, g1, vy, vx, Sy, Sx, lcm):
    """The kernels' rule; g = (first scan position of the group, position mod S_x).  None where
    the kernels fall back to the full index."""
    d64 = (64 * vx % Sx) * (lcm // Sx)
    if g1[0] == g0[0] + 64 and g1[1] == g0[1] + 64:
        return (m0 + d64) % lcm
    if g1[0] == g0[0] + 64 and g1[1] == g0[1] + 64 - Sx:
        return ((m0 + d64) % lcm + vy * (lcm // Sy)) % lcm
    return None


@pytest.mark.parametrize("Sy,Sx", [(128, 128), (17, 23), (40, 40), (33, 40), (8, 96), (64, 50)])
def test_stepped_index_equals_the_full_index(Sy, Sx):
    """Every frequency (as integer arrays) and every pair of groups 64 positions apart."""
    lcm = Sy * Sx // math.gcd(Sy, Sx)
    vy, vx = (a.astype(np.int64).ravel() for a in np.meshgrid(np.arange(Sy), np.arange(Sx),
                                                              indexing="ij"))
    stepped = 0
    for s0 in range(0, Sy * Sx - 64, 16):
        s1 = s0 + 64
        m0 = full_index(s0, vy, vx, Sy, Sx, lcm)
        m1 = stepped_index(m0, (s0, s0 % Sx), (s1, s1 % Sx), vy, vx, Sy, Sx, lcm)
        if m1 is None:
            continue
        stepped += 1
        assert np.array_equal(m1, full_index(s1, vy, vx, Sy, Sx, lcm)), s0
    if Sx >= 33:   # some step taken along a row or across a wrap
        assert stepped > 0


@pytest.mark.parametrize("Sy,Sx", [(128, 128), (40, 40), (64, 50)])
def test_index_gives_the_scan_phase(Sy, Sx):
    lcm = Sy * Sx // math.gcd(Sy, Sx)
    rng = np.random.default_rng(7)
    for _ in range(200):
        vy, vx = int(rng.integers(Sy)), int(rng.integers(Sx))
        s = int(rng.integers(Sy * Sx))
        sy, sx = divmod(s, Sx)
        m = full_index(s, vy, vx, Sy, Sx, lcm)
        direct = np.exp(-2j * np.pi * (vy * sy / Sy + vx * sx / Sx))
        assert abs(np.exp(-2j * np.pi * m / lcm) - direct) < 1e-12


def test_row_wrap_rule_is_taken_on_a_raster_scan():
    # 128-wide scan: a 64-frame stage starting mid-row wraps into the next row
    Sy, Sx = 128, 128
    lcm = 128
    s0 = 5 * Sx + 64
    g0, g1 = (s0, s0 % Sx), (s0 + 64, (s0 + 64) % Sx)
    assert g1[1] == g0[1] + 64 - Sx
    for vy, vx in [(0, 0), (1, 0), (0, 1), (77, 31), (127, 127)]:
        m0 = full_index(s0, vy, vx, Sy, Sx, lcm)
        assert stepped_index(m0, g0, g1, vy, vx, Sy, Sx, lcm) == full_index(s0 + 64, vy, vx, Sy, Sx, lcm)
