"""Pins of the oracle's synthetic mesh map to values worked out by hand.

The shear x' = x + amp sin(2 pi y) sin(2 pi z) (2D: x' = x + amp sin(2 pi y))
at points where the sines are 0 or +-1 gives exact values, so a wrong
amplitude, argument, sign or axis in ``shear_map`` fails here, which the
constant-Jacobian and volume checks (true for any x' = x + f(y, z)) cannot
see.  ``StructuredMesh.physical`` is pinned the same way through an element
whose reference corner lands on such a point.
"""
import numpy as np
import pytest

from oracle.geometry import StructuredMesh, shear_map


@pytest.mark.parametrize("X,expect", [
    ((0.0, 0.25, 0.25), (0.05, 0.25, 0.25)),      # sin(pi/2) sin(pi/2) = 1
    ((0.3, 0.25, 0.75), (0.25, 0.25, 0.75)),      # sin(pi/2) sin(3 pi/2) = -1
    ((0.7, 0.125, 0.5), (0.7, 0.125, 0.5)),       # sin(pi) = 0
    ((0.5, 0.75, 0.75), (0.55, 0.75, 0.75)),      # (-1)(-1) = 1
])
def test_shear_map_3d_closed_form(X, expect):
    y = shear_map(3, 0.05, np.array(X))
    np.testing.assert_allclose(y, expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("X,expect", [((0.1, 0.25), (0.15, 0.25)), ((0.1, 0.75), (0.05, 0.75)),
                                      ((0.9, 0.5), (0.9, 0.5))])
def test_shear_map_2d_closed_form(X, expect):
    np.testing.assert_allclose(shear_map(2, 0.05, np.array(X)), expect, rtol=0, atol=1e-15)


def test_physical_places_elements_on_the_map():
    # 4^3 elements of width 1/4: element (ex, ey, ez) = (1, 1, 2) has its
    # reference corner (-1, -1, -1) at (1/4, 1/4, 1/2) and (+1, -1, -1) at
    # (1/2, 1/4, 1/2); sin(pi/2) sin(pi) = 0 there, and at the corner
    # (-1, -1, +1) = (1/4, 1/4, 3/4): sin(pi/2) sin(3 pi/2) = -1.
    m = StructuredMesh(3, 4, 2, amp=0.05)
    e = 1 + 4 * (1 + 4 * 2)
    ref = np.array([[-1.0, -1, -1], [1, -1, -1], [-1, -1, 1]])
    x = m.physical(np.array([e]), ref)[0]
    np.testing.assert_allclose(x, [[0.25, 0.25, 0.5], [0.5, 0.25, 0.5], [0.2, 0.25, 0.75]], rtol=0, atol=1e-15)
