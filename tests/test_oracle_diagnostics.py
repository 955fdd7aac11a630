"""Pins of the oracle's two diagnostics against hand-computed values.

* The steady-state criterion of Sec. 4: the relative change of u and T over a
  lag, with u measured by the Euclidean norm of each node's velocity summed
  over the nodes and T by its absolute value summed over the nodes, both
  divided by the norm of the NEW field.  The 3 x 2 fields below are built
  from Pythagorean triples so that every norm is an integer; the expected
  ratios are written as the hand sums.  Each plausible misreading (per
  component absolute values, squared norms, root of the ratio of squares, the
  old field in the denominator, signed sums for T) gives a different number.
* The Nusselt number of Eq. (Eq:AvNuss): Nu(j) = -L (dT/dn)_wall / (Th - Tc)
  along the wall-normal axis, with the mean as the trapezoid rule over the
  wall's nodes divided by (nodes - 1).  On a temperature field quadratic in
  the distance from the wall the second-order one-sided difference is exact,
  so Nu(j) is known in closed form from the field's linear coefficient b(j)
  (a first-order difference would add the quadratic coefficient); with
  b(j) = j^2 the trapezoid mean has the closed form
  (H + 1)(2H + 1)/6 - H/2 (H = nodes - 1), which differs from the plain mean
  H(2H + 1)/6 and from the integral H^2/3.  A 7 x 5 lattice with Th - Tc = 2
  catches transposed indices and a wrong normaliser.
"""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import workloads as W

# velocity (ux, uy) per node and its Euclidean norm:
#   (3, 4) 5, (5, 12) 13, (8, 15) 17, (0, 0) 0, (-7, 24) 25, (20, 21) 29  -> sum 89
UX = np.array([[3.0, 5.0, 8.0], [0.0, -7.0, 20.0]])
UY = np.array([[4.0, 12.0, 15.0], [0.0, 24.0, 21.0]])
# change over the lag (new - old) and its norm:
#   (3, 4) 5, (0, 0) 0, (-6, 8) 10, (0, -1) 1, (5, -12) 13, (8, 15) 17   -> sum 46
DUX = np.array([[3.0, 0.0, -6.0], [0.0, 5.0, 8.0]])
DUY = np.array([[4.0, 0.0, 8.0], [-1.0, -12.0, 15.0]])
# temperature: |T| sums to 0.5 + 0.25 + 1 + 0 + 2 + 1.5 = 5.25;
# |dT| sums to 0.25 + 0.5 + 0.25 + 0.125 + 0.75 + 1 = 2.875
T = np.array([[0.5, -0.25, 1.0], [0.0, 2.0, -1.5]])
DT = np.array([[0.25, -0.5, 0.25], [0.125, -0.75, 1.0]])


def test_residual_hand_computed():
    res_u, res_T = oracle.residual(UX, UY, T, UX - DUX, UY - DUY, T - DT)
    assert res_u == pytest.approx(46.0 / 89.0, rel=1e-15)
    assert res_T == pytest.approx(2.875 / 5.25, rel=1e-15)
    # the misreadings it must not match
    wrong_u = [62.0 / 119.0,                       # per-component absolute values
               584.0 / 1949.0,                     # squared norms
               np.sqrt(584.0 / 1949.0)]            # root of the ratio of squares
    for w in wrong_u:
        assert abs(res_u - w) > 1e-3
    wrong_T = [0.125 / 1.75,                       # signed sums
               2.875 / 6.625,                      # old field in the denominator
               np.sqrt(1.953125 / 7.5625)]         # L2 norms
    for w in wrong_T:
        assert abs(res_T - w) > 1e-3


def test_residual_zero_and_scale_invariant():
    assert oracle.residual(UX, UY, T, UX, UY, T) == (0.0, 0.0)
    a = oracle.residual(UX, UY, T, UX - DUX, UY - DUY, T - DT)
    b = oracle.residual(8 * UX, 8 * UY, 4 * T, 8 * (UX - DUX), 8 * (UY - DUY), 4 * (T - DT))
    assert b[0] == pytest.approx(a[0], rel=1e-15) and b[1] == pytest.approx(a[1], rel=1e-15)


NX, NY = 7, 5
TH, TC = 1.5, -0.5          # Th - Tc = 2
L = NX - 1                  # L = nx - 1 (wall nodes are lattice nodes)


def _quadratic_field(side):
    """T = 0.3 + b(j) d + 0.7 d^2 with d the distance from `side` and j the
    index along it, b(j) = j^2."""
    yy, xx = np.mgrid[0:NY, 0:NX].astype(float)
    d, j = {"W": (xx, yy), "E": (NX - 1 - xx, yy), "S": (yy, xx), "N": (NY - 1 - yy, xx)}[side]
    return 0.3 + j ** 2 * d + 0.7 * d ** 2


@pytest.mark.parametrize("side", ["W", "E", "S", "N"])
def test_nusselt_exact_on_quadratic_profile(side):
    p = W.cavity(NX, 1e3, 1e-2, 0.6, ny=NY, Th=TH, Tc=TC)
    o = oracle.Oracle(p)
    mean, loc = o.nusselt(side, T=_quadratic_field(side))
    n = NY if side in ("W", "E") else NX
    j = np.arange(n, dtype=float)
    # dT/dd at the wall is b(j) = j^2; the derivative along the +x (+y) axis
    # is +b on W (S) and -b on E (N); Nu = -L (dT/daxis) / (Th - Tc)
    sign = -1.0 if side in ("W", "S") else 1.0
    expect_loc = sign * L * j ** 2 / (TH - TC)
    assert np.allclose(loc, expect_loc, rtol=1e-13, atol=1e-12)
    H = n - 1
    trap = (H + 1) * (2 * H + 1) / 6.0 - H / 2.0     # trapezoid sum of j^2 over H
    assert mean == pytest.approx(sign * L * trap / (TH - TC), rel=1e-13)
    # neither the plain mean nor the exact integral of j^2
    for wrong in (H * (2 * H + 1) / 6.0, H * H / 3.0):
        assert abs(mean - sign * L * wrong / (TH - TC)) > 1e-3 * abs(mean)
