"""D3Q19 lattice for the oracle (test infrastructure only).

The paper names the LBM basis (distribution G_i, weights omega_i, lattice
speed C; Sec. 2.3.2, Eq. of the interpolated bounce-back) but not the lattice.
Reading A23: the standard D3Q19 BGK lattice with C = 1, c_s^2 = 1/3.

Direction order: 0 = rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the twelve edge
diagonals, each followed by its opposite.  So for i >= 1 the opposite of an
odd i is i+1 and of an even i is i-1.
"""
import numpy as np

E = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0),
    (0, 1, 0), (0, -1, 0),
    (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0),
    (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1),
    (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1),
    (0, 1, -1), (0, -1, 1),
], dtype=np.int64)

W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12, dtype=np.float64)

OPP = np.array([0] + [i + 1 if i % 2 == 1 else i - 1 for i in range(1, 19)], dtype=np.int64)

Q = 19
CS2 = 1.0 / 3.0
