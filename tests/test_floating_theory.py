"""The stability helper of the floating-cube test against the angles the
paper gives for a square (Sec. 3.2.2) and against the mirror symmetry
s <-> 1 - s (no GPU)."""
import math

import pytest

from floating import immersed, stable_heel, stable_heel_compressible


def test_square_stable_heels_of_the_paper():
    assert stable_heel(0.25) == pytest.approx(math.degrees(math.atan(0.5)), abs=0.02)
    assert stable_heel(0.75) == pytest.approx(math.degrees(math.atan(0.5)), abs=0.02)
    assert stable_heel(0.5) == pytest.approx(45.0, abs=0.02)


def test_mirror_symmetry_and_upright_square():
    for s in (0.23, 0.27, 0.4):
        assert stable_heel(s) == pytest.approx(stable_heel(1.0 - s), abs=0.05)
    bx, depth = immersed(0.5, 0.0)
    assert abs(bx) < 1e-12 and depth == pytest.approx(0.25, abs=1e-9)


def test_denser_liquid_lightens_the_box():
    """A liquid denser than 1 at depth makes the 3/4 box float like a lighter
    one, which moves its stable heel towards 45 deg, and the 1/4 box's below
    atan(1/2)."""
    g, side = 7.5e-4, 16.0
    assert stable_heel_compressible(0.75, side, g) > stable_heel(0.75) + 1.5
    assert stable_heel_compressible(0.25, side, g) < stable_heel(0.25)
    assert stable_heel_compressible(0.5, side, g) == pytest.approx(45.0, abs=0.02)
