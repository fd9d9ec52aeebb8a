"""The allocation-free mass-property entry point (for callers whose device
memory is reserved by another allocator, or who cannot take the
synchronisation of a cudaFree) must give what mi_delbm_add_particle computes
for the same particle, call after call: two calls in a row, the second on a
smaller ball table, so that scratch left over from the first call would show.
It must also give the FP64 oracle's quadrature at another spacing, and NaN
outputs, promptly, for a particle with no solid volume at the spacing and for
a grid beyond its limits.
"""
import time

import numpy as np
import pytest

from oracle import metaball
from paper_2209_10411_gb300 import scenes
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu


def _existing_entry_point(B, c, k, density):
    """mass, volume, centroid and inertia from mi_delbm_add_particle (which
    allocates its quadrature scratch through the handle)."""
    sim = B.Simulation(64, 64, 64, tau=0.8, max_balls=8192)
    pos = np.array([32.0, 32.0, 32.0])
    sim.add_particle(c, k, density, 0.5, pos, (1.0, 0.0, 0.0, 0.0))
    sh = sim.get_particle_shape(0)
    centroid = c[0] - sh["centers"][0]
    sim.close()
    return sh["mass"], sh["volume"], centroid, sh["inertia"]


def test_noalloc_matches_add_particle_two_calls():
    import torch
    B = binding()
    rng = np.random.default_rng(2024)
    big_c, big_k, _ = scenes.cobble(rng, n_range=(30, 30), semi=(10.0, 14.0), k_range=(4.0, 16.0))
    small_c, small_k, _ = scenes.blob_4(rng)
    stream = torch.cuda.current_stream()
    for c, k, density in [(big_c, big_k, 2.5), (small_c, small_k, 1.7)]:
        balls = torch.tensor(np.c_[c, k], dtype=torch.float64, device="cuda")
        out = torch.full((14,), float("nan"), dtype=torch.float64, device="cuda")
        B.mass_properties_noalloc(balls.data_ptr(), len(k), density, 0.25, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        mass, vol, cen, inertia = _existing_entry_point(B, c, k, density)
        assert np.isfinite(got).all()
        assert abs(got[1] - vol) <= 1e-9 * vol
        assert abs(got[0] - mass) <= 1e-9 * mass
        assert np.allclose(got[2:5], cen, rtol=0, atol=1e-9 * max(1.0, np.abs(c).max()))
        assert np.allclose(got[5:].reshape(3, 3), inertia, rtol=1e-8, atol=1e-8 * np.abs(inertia).max())


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    B = binding()
    balls = torch.zeros((4097, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(14, dtype=torch.float64, device="cuda")
    with pytest.raises(B.MiDelbmError) as ei:
        B.mass_properties_noalloc(balls.data_ptr(), 4097, 1.0, 0.25, out.data_ptr())
    assert ei.value.status == B.MI_EINVAL and "4096" in str(ei.value)


def _noalloc(B, c, k, density, spacing):
    import torch
    stream = torch.cuda.current_stream()
    balls = torch.tensor(np.c_[c, k], dtype=torch.float64, device="cuda")
    out = torch.zeros(14, dtype=torch.float64, device="cuda")
    B.mass_properties_noalloc(balls.data_ptr(), len(k), density, spacing, out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_oracle_at_half_spacing():
    """The 30-ball cobble at spacing 1/2 against the oracle's midpoint
    quadrature of f >= 1 (reading A15): the same samples decided the same way
    (FP32 field with an FP64 re-check near f = 1), so the same count; the
    moments within rounding of the two summation orders."""
    B = binding()
    rng = np.random.default_rng(2024)
    c, k, _ = scenes.cobble(rng, n_range=(30, 30), semi=(10.0, 14.0), k_range=(4.0, 16.0))
    got = _noalloc(B, c, k, 2.5, 0.5)
    ref = metaball.mass_properties(c, k, 2.5, h=0.5)
    assert got[1] == pytest.approx(ref["volume"], rel=1e-12)
    assert got[0] == pytest.approx(ref["mass"], rel=1e-12)
    assert np.allclose(got[2:5], ref["centroid"], rtol=0, atol=1e-9)
    assert np.allclose(got[5:].reshape(3, 3), ref["inertia"], rtol=1e-9, atol=1e-9 * np.abs(ref["inertia"]).max())


def test_noalloc_nan_without_volume_or_beyond_the_grid_limit():
    B = binding()
    # one ball of radius 0.1 sampled at spacing 1: the only sample is outside
    got = _noalloc(B, np.zeros((1, 3)), np.array([0.01]), 1.0, 1.0)
    assert np.isnan(got).all()
    # a cobble at spacing 1e-4: about 7e5 samples per axis, not run
    rng = np.random.default_rng(7)
    c, k, _ = scenes.cobble(rng)
    t0 = time.perf_counter()
    got = _noalloc(B, c, k, 2.5, 1e-4)
    assert time.perf_counter() - t0 < 5.0
    assert np.isnan(got).all()
    # and the next call on a valid table is unaffected
    got = _noalloc(B, c, k, 2.5, 0.5)
    ref = metaball.mass_properties(c, k, 2.5, h=0.5)
    assert got[1] == pytest.approx(ref["volume"], rel=1e-12)
