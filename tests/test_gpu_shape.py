"""GPU parity of the shape descriptors (Sec. 3; mi_shape_descriptors)
against the oracle, through the C-ABI.

Bars: the solid-cell count is an integer both sides take in FP32 with the
same single roundings: equal; the volume follows; the surface (FP32 band sums
against FP64) within 1e-4; the principal axes within 1e-4 (up to sign); the
extents and the projected area come from a second grid whose orientation is
the axes' (FP32 on the GPU, FP64 eigenvectors in the oracle), so cells at
the boundary may differ: extents within one cell h, projected area within
2 %; a sphere gives the sphere's values."""
import numpy as np
import pytest

from oracle import shape
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu


def _models(seed, count):
    rng = np.random.default_rng(seed)
    out = [(np.zeros((1, 3)), np.array([9.0]))]
    for _ in range(count - 1):
        c, k, _ = scenes.cobble(rng, n_range=(4, 12), semi=(3.0, 6.0), k_range=(1.0, 4.0))
        out.append((c, k))
    return out


@pytest.mark.parametrize("h", [1.0 / 8, 1.0 / 5])
def test_descriptors_match_oracle(h):
    B = binding()
    models = _models(3, 6)
    got = B.shape_descriptors(models, h)
    for (c, k), g in zip(models, got):
        o = shape.descriptors(c, k, h)
        assert int(g["cells"]) == o["cells"]
        assert g["volume"] == pytest.approx(o["volume"], rel=1e-12)
        assert g["surface"] == pytest.approx(o["surface"], rel=1e-4)
        ev = o["eigenvalues"]
        for r in range(3):
            gap = min(abs(ev[r] - ev[q]) for q in range(3) if q != r) / ev[0]
            if gap > 1e-2:  # an axis is defined (to within FP32 moments) only away from degeneracy
                assert abs(abs(float(np.dot(g["axes"][r], o["axes"][:, r]))) - 1.0) < 1e-4, r
        assert np.allclose([g["l_long"], g["l_int"], g["l_short"]], o["lengths"], atol=h * 1.01)
        assert g["projected_area"] == pytest.approx(o["projected_area"], rel=2e-2)
        assert g["sphericity"] == pytest.approx(o["sphericity"], rel=1e-4)
        assert g["csf"] == pytest.approx(o["csf"], abs=3 * h / o["lengths"][2])


def test_sphere_and_batch_independence():
    B = binding()
    models = _models(4, 5)
    got = B.shape_descriptors(models, 1.0 / 16)
    s = got[0]
    assert s["sphericity"] == pytest.approx(1.0, abs=1e-2)
    assert s["csf"] == pytest.approx(1.0, abs=0.05)
    assert s["volume"] == pytest.approx(4.0 / 3.0 * np.pi * 27.0, rel=5e-3)
    one = B.shape_descriptors([models[2]], 1.0 / 16)[0]
    assert one["cells"] == got[2]["cells"] and one["volume"] == got[2]["volume"]
