"""Solid flagging of nodes whose field lies in the FP32 guard band of the
iso-value (Sec. 2.1, Eq. 1: a node is solid when f >= 1).  The flag kernel
decides |f - 1| <= 1e-4 again in FP64, the whole warp forming one node's
terms and summing them in ball order; the owners must equal the FP64
oracle's bit for bit.

A one-ball particle of k = 25 centred on a lattice node, unrotated, has the
30 integer points at distance 5 exactly on its surface (f = 1: solid);
k = 25 (1 - 3e-7) moves them just outside and k = 25 (1 + 3e-7) just
inside, well within the guard band of the FP32 pass, so every one of them
takes the FP64 path."""
import numpy as np
import pytest

from oracle import metaball
from tests.gpu_helpers import binding

pytestmark = pytest.mark.gpu

SHAPE = (32, 30, 28)
POS = np.array([15.0, 14.0, 13.0])


def _owners_gpu(B, centers, k):
    mp = metaball.mass_properties(centers, k, 2.5)
    with B.Simulation(*SHAPE, tau=0.8) as sim:
        sim.add_particle(centers, k, 2.5, 0.5, POS, np.array([1.0, 0.0, 0.0, 0.0]),
                         mass_props={"mass": mp["mass"], "volume": mp["volume"], "inertia": mp["inertia"]})
        sim.step_phases(B.PHASE_FLAG)
        _, own = sim.node_classes()
    own = own.astype(np.int64)
    own[own == 0xFFFFFFFF] = -1
    return own


def test_surface_nodes_decided_in_fp64():
    B = binding()
    centers = np.zeros((1, 3))
    counts = []
    for k0 in (25.0 * (1.0 - 3e-7), 25.0, 25.0 * (1.0 + 3e-7)):
        k = np.array([k0])
        ref = metaball.flag_nodes(SHAPE, [{"centers": centers, "k": k, "pos": POS,
                                           "quat": np.array([1.0, 0.0, 0.0, 0.0])}])
        got = _owners_gpu(B, centers, k)
        assert np.array_equal(got, ref), (k0, int((got != ref).sum()))
        counts.append(int((ref >= 0).sum()))
    # the 30 nodes at distance exactly 5 are solid from k = 25 on
    assert counts[1] - counts[0] == 30 and counts[2] == counts[1], counts


def test_two_balls_near_the_surface():
    """Two balls whose summed field puts nodes at non-integer distances near
    f = 1 (some of them inside the guard band); owners bit-exact."""
    B = binding()
    centers = np.array([[-1.25, 0.0, 0.0], [1.25, 0.5, 0.0]])
    k = np.array([9.0, 7.0])
    ref = metaball.flag_nodes(SHAPE, [{"centers": centers, "k": k, "pos": POS,
                                       "quat": np.array([1.0, 0.0, 0.0, 0.0])}])
    got = _owners_gpu(B, centers, k)
    assert np.array_equal(got, ref), int((got != ref).sum())
