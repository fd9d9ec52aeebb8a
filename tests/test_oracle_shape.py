"""Pins of the shape-descriptor oracle (Sec. 3 definitions, readings D1-D5):
a single ball is a sphere (volume, surface, sphericity 1, axis lengths,
projected area and CSF 1 within the quadrature's resolution), the metaball
scale law (centres x2, k x4, spacing x2) scales the quadratures exactly, and
an elongated two-ball particle orders its axes and has CSF below 1."""
import numpy as np
import pytest

from oracle import shape


def test_single_ball_is_a_sphere():
    k = 9.0
    d = shape.descriptors(np.zeros((1, 3)), np.array([k]), 1.0 / 16)
    r = np.sqrt(k)
    assert d["volume"] == pytest.approx(4.0 / 3.0 * np.pi * r ** 3, rel=5e-3)
    assert d["surface"] == pytest.approx(4.0 * np.pi * k, rel=1e-2)
    assert d["sphericity"] == pytest.approx(1.0, abs=1e-2)
    assert np.allclose(d["lengths"], 2 * r, atol=2.0 / 16)
    assert d["projected_area"] == pytest.approx(np.pi * k, rel=2e-2)
    assert d["csf"] == pytest.approx(1.0, abs=0.05)
    assert d["d_n"] == pytest.approx(2 * r, rel=5e-3)


def test_scale_law():
    c = np.array([[-1.0, 0.2, 0.0], [1.2, -0.1, 0.3]])
    k = np.array([3.0, 2.0])
    a = shape.descriptors(c, k, 1.0 / 8)
    b = shape.descriptors(2.0 * c, 4.0 * k, 1.0 / 4)
    assert a["cells"] == b["cells"]
    assert b["volume"] == pytest.approx(8.0 * a["volume"], rel=1e-12)
    assert b["surface"] == pytest.approx(4.0 * a["surface"], rel=1e-9)
    assert np.allclose(b["lengths"], 2.0 * a["lengths"], atol=2 * 0.25)
    assert b["sphericity"] == pytest.approx(a["sphericity"], rel=1e-9)


def test_elongated_particle():
    c = np.array([[-2.5, 0.0, 0.0], [0.0, 0.0, 0.0], [2.5, 0.0, 0.0]])
    k = np.array([2.0, 2.0, 2.0])
    d = shape.descriptors(c, k, 1.0 / 8)
    L = d["lengths"]
    assert L[0] > 1.4 * L[1] and abs(L[1] - L[2]) <= 2.0 / 8
    assert abs(abs(d["axes"][0, 0]) - 1.0) < 1e-6  # the longest axis is x
    assert 0.4 < d["csf"] < 0.9 and d["sphericity"] < 1.0
    # the projection along the shortest axis holds the long and intermediate axes
    assert d["projected_area"] > 0.6 * np.pi / 4 * L[0] * L[1]
