"""The algorithmic work bench.py divides by a kernel's time, against closed
forms: sum_{n<p} (2n+1)^2 = p (2p-1)(2p+1)/3 (the rotation blocks of degrees
below p, Sec. 3.3) and sum_{|m|<p} (p-|m|)^2 = p (2p^2+1)/3 (the coaxial
blocks), 8 real flops per complex multiply-accumulate."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench


def test_rotation_and_coaxial_counts_match_closed_forms():
    for p in (1, 2, 12, 89, 159):
        rot = p * (2 * p - 1) * (2 * p + 1) // 3
        cox = p * (2 * p * p + 1) // 3
        assert bench.rot_flops(p, p) == 8.0 * 2 * rot
        assert bench.coax_flops(p, p) == 8.0 * cox
        assert bench.rcr_flops(p, p) == 8.0 * (2 * rot + cox)


def test_unequal_orders():
    # M2M-like translation 3 -> 5: rotations of degrees < 3 and < 5, coaxial
    # blocks (5-|m|)(3-|m|) for |m| < 3
    assert bench.rot_flops(5, 3) == 8.0 * ((1 + 9 + 25) + (1 + 9 + 25 + 49 + 81))
    assert bench.coax_flops(5, 3) == 8.0 * (5 * 3 + 2 * (4 * 2) + 2 * (3 * 1))
