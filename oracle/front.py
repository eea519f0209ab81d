"""Position of the phase interface measured on a temperature field (test
infrastructure only, see ``oracle/__init__.py``).

The paper plots the interface position (Sec. 6.1) without defining how it is
read off the lattice.  The reading used here, for every lattice line that
starts at a given wall (rows for the W and E walls, columns for S and N),
with node 0 on the wall:

* first zero: the first sign change of theta from the wall's sign, linearly
  interpolated between the two nodes around it, x_f = (i - 1) + t_{i-1} /
  (t_{i-1} - t_i) in node units; 0 if theta is 0 on the wall node; n - 1 if
  the sign never changes;
* integrated: the wall side's phase fraction summed along the line minus the
  half cell of the wall node, sum_i phi(theta_i) - 1/2 for a wall node above
  the melting point, sum_i (1 - phi(theta_i)) - 1/2 otherwise
  (phi = (1 + tanh(theta/delta))/2, Sec. 4.1).

Both are returned per line and as the mean over the lines.  Plain loops, in
FP64: this is the definition written out.
"""
from __future__ import annotations

import math

import numpy as np


def _lines(theta, wall):
    """The lattice lines that start at `wall` (0 W, 1 E, 2 S, 3 N), node 0 on
    the wall; theta has shape (ny, nx)."""
    t = np.asarray(theta, dtype=np.float64)
    if t.ndim == 1:
        t = t[None, :]
    if wall == 0:
        return t
    if wall == 1:
        return t[:, ::-1]
    if wall == 2:
        return t.T
    if wall == 3:
        return t[::-1, :].T
    raise ValueError("wall must be 0..3")


def first_zero(line):
    """First sign change from the wall node's sign, node units."""
    t0 = float(line[0])
    if t0 == 0.0:
        return 0.0
    for i in range(1, len(line)):
        ti = float(line[i])
        if (t0 > 0.0 and ti <= 0.0) or (t0 < 0.0 and ti >= 0.0):
            a = float(line[i - 1])
            return (i - 1) + a / (a - ti)
    return float(len(line) - 1)


def integrated(line, delta):
    """Wall-side phase fraction summed along the line, minus the wall half cell."""
    hot = float(line[0]) > 0.0
    s = 0.0
    for v in line:
        ph = 0.5 * (1.0 + math.tanh(float(v) / delta))
        s += ph if hot else 1.0 - ph
    return s - 0.5


def front_position(theta, delta, wall=0):
    """(mean first zero, mean integrated, per-line first zeros, per-line integrated)."""
    lines = _lines(theta, wall)
    fz = np.array([first_zero(l) for l in lines])
    it = np.array([integrated(l, delta) for l in lines])
    return float(fz.mean()), float(it.mean()), fz, it
