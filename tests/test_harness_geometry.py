"""The cone of the adjoint's observable, as the tests define it (no GPU).

The GPU adjoint's J equals the cone sum of tests/harness.py to 1e-13
(tests/test_gpu_adjoint.py); this pins that cone to its closed form: the cells
whose centres it holds fill the volume of a spherical sector,
V = (2 pi / 3) r^3 (1 - cos theta), to the discretisation error of the cell
boundary, for any axis.  A mistaken reading (full instead of half angle,
degrees as radians, diameter for radius, a cone opening backwards) is off by a
factor of 3 or more.
"""
import math

import numpy as np
import pytest

from harness import cone_mask


@pytest.mark.parametrize("axis", [(1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (1.0, 1.0, 1.0)])
@pytest.mark.parametrize("half_angle", [30.0, 60.0])
def test_cone_holds_the_volume_of_a_spherical_sector(axis, half_angle):
    dx, r = 0.1, 3.0
    n = (64, 64, 64)
    apex = (0.013, -0.021, 0.007)           # off the cell lattice
    got = cone_mask(n, dx, apex, axis, half_angle, r).sum() * dx ** 3
    want = 2.0 * math.pi / 3.0 * r ** 3 * (1.0 - math.cos(math.radians(half_angle)))
    assert abs(got / want - 1.0) < 0.005, (got, want)   # measured <= 0.13 %


def test_cone_opens_along_its_axis():
    n, dx = (40, 40, 40), 0.1
    m = cone_mask(n, dx, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0))
    x = (np.arange(n[0]) + 0.5 - n[0] / 2) * dx
    assert m.any() and np.all(x[np.nonzero(m)[2]] > 0.0)
