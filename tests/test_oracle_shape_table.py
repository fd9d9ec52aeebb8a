"""Pin of the shape-descriptor oracle against the descriptors the paper
prints for the particles of its DKT study (Sec. 3; tests/golden/
dkt_particle_shapes.txt).

With d_n the volume-equivalent diameter, d_s = sqrt(4 A_p / pi) from the
projection along the shortest axis, and CSF = L_short / sqrt(L_int L_long)
(readings D4, D5), an ellipsoid of semi-axes a >= b >= c has
d_n / d_s = (abc)^(1/3) / (ab)^(1/2) = CSF^(1/3) exactly.  Every row of the
printed table obeys this within 0.9 %, so a metaball body of the same kind
(control points moved apart along three axes, as the paper builds P2-P8)
must obey it within the same margin plus the quadrature's resolution.  A
projection along the wrong axis, a CSF with the wrong numerator or a
diameter off by a factor fails by far more."""
import os

import numpy as np
import pytest

from oracle import shape

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dkt_particle_shapes.txt")


def _table():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, phi, r, csf = line.split()
        rows.append((name, float(phi), float(r), float(csf)))
    return rows


def test_printed_table_obeys_the_ellipsoid_relation():
    rows = _table()
    assert len(rows) == 9
    for name, phi, r, csf in rows:
        assert 0.0 < csf <= 1.0 and 0.0 < phi <= 1.0
        assert r == pytest.approx(csf ** (1.0 / 3.0), rel=1e-2), name


def _spread_model(s):
    """Six unit control points at +-s, +-0.6 s, +-0.3 s on the three axes."""
    a, b, c = s, 0.6 * s, 0.3 * s
    C = np.array([[a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0], [0, 0, c], [0, 0, -c]], dtype=float)
    return C, np.ones(6)


def test_oracle_follows_the_table_relation_over_its_csf_range():
    table_csf = [csf for _, _, _, csf in _table()]
    seen = []
    for s in (0.0, 0.8, 1.6, 2.4, 2.8):
        C, k = _spread_model(s)
        d = shape.descriptors(C, k, 1.0 / 10)
        r = d["d_n"] / d["d_s"]
        assert r == pytest.approx(d["csf"] ** (1.0 / 3.0), rel=1e-2), s
        assert d["sphericity"] <= 1.0 + 1e-2
        L = d["lengths"]
        assert L[0] >= L[1] >= L[2]
        seen.append(d["csf"])
    # moving the control points apart lowers the CSF monotonically, across
    # the whole range of the printed particles
    assert all(x > y for x, y in zip(seen, seen[1:]))
    assert seen[0] >= max(table_csf) - 1e-2 and seen[-1] <= min(table_csf) + 1e-2
