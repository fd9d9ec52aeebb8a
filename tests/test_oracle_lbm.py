"""Pins of the oracle's lattice Boltzmann part against the lattice definition,
conservation laws and closed-form flows (no GPU).

Each test is chosen so that a plausible mistake in the oracle fails it: a wrong
weight or velocity (isotropy), a wrong equilibrium coefficient (moments), a
swapped axis or sign in streaming (delta advection, Couette), a lost term in
the bounce-back (mass conservation, Couette), a wrong Guo term (momentum
gain, Poiseuille curvature).
"""
import itertools

import numpy as np
import pytest

from oracle import lbm
from oracle.d3q19 import E, OPP, Q, W

TAU = 0.8


def test_lattice_isotropy():
    # D3Q19 moments up to fourth order: the lattice definition.
    Ef = E.astype(float)
    assert abs(W.sum() - 1.0) < 1e-15
    assert np.allclose((W[:, None] * Ef).sum(0), 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", W, Ef, Ef)
    assert np.allclose(M2, np.eye(3) / 3.0, atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", W, Ef, Ef, Ef)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", W, Ef, Ef, Ef, Ef)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(M4, iso, atol=1e-15)
    for i in range(Q):
        assert (E[OPP[i]] == -E[i]).all()
    assert len({tuple(e) for e in E}) == 19
    assert all(np.abs(e).sum() <= 2 for e in E)


def test_equilibrium_moments_closed_form():
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.1 * rng.standard_normal((3, 4, 5))
    u = 0.05 * rng.standard_normal((3, 3, 4, 5))
    feq = lbm.equilibrium(rho, u)
    Ef = E.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=1e-14)
    mom = np.einsum("ia,i...->a...", Ef, feq)
    assert np.allclose(mom, rho * u, atol=1e-15)
    # second moment of the second-order equilibrium: rho (u u + I/3)
    P = np.einsum("ia,ib,i...->ab...", Ef, Ef, feq)
    expect = rho * (np.einsum("a...,b...->ab...", u, u) + np.eye(3)[:, :, None, None, None] / 3.0)
    assert np.allclose(P, expect, atol=1e-14)


def _random_state(shape, seed=0, amp=0.05):
    rng = np.random.default_rng(seed)
    return W.reshape((Q, 1, 1, 1)) * (1.0 + amp * rng.standard_normal((Q,) + shape))


def test_collide_conserves_mass_and_momentum():
    f = _random_state((4, 5, 6))
    fp = lbm.collide(f, TAU)
    Ef = E.astype(float)
    assert np.allclose(fp.sum(0), f.sum(0), rtol=0, atol=1e-14)
    assert np.allclose(np.einsum("ia,i...->a...", Ef, fp), np.einsum("ia,i...->a...", Ef, f),
                       rtol=0, atol=1e-15)
    # BGK relaxes the non-equilibrium part by exactly (1 - 1/tau)
    rho, u = lbm.moments(f)
    feq = lbm.equilibrium(rho, u)
    assert np.allclose(fp - feq, (1 - 1 / TAU) * (f - feq), atol=1e-15)


def test_guo_forcing_momentum_gain():
    # Guo forcing adds exactly F to the momentum per collision and no mass.
    f = _random_state((3, 4, 5), seed=2)
    F = np.array([1e-4, -2e-4, 3e-4])
    fp = lbm.collide(f, TAU, force=F)
    Ef = E.astype(float)
    dm = np.einsum("ia,i...->a...", Ef, fp) - np.einsum("ia,i...->a...", Ef, f)
    assert np.allclose(dm, F[:, None, None, None], atol=1e-15)
    assert np.allclose(fp.sum(0), f.sum(0), atol=1e-14)


def test_stream_moves_each_population_by_its_velocity():
    # A single unit population at one node ends up at x + e_i (periodic box).
    shape = (5, 6, 7)
    for i in range(Q):
        f = np.zeros((Q,) + shape)
        x, y, z = 3, 2, 1
        f[i, z, y, x] = 1.0
        g = lbm.stream_pull(f, periodic=(True, True, True))
        dst = ((z + E[i, 2]) % 5, (y + E[i, 1]) % 6, (x + E[i, 0]) % 7)
        assert g[i][dst] == 1.0
        assert g.sum() == 1.0


def test_stream_periodic_is_permutation():
    f = _random_state((5, 6, 7), seed=3)
    g = lbm.stream_pull(f, periodic=(True, True, True))
    for i in range(Q):
        assert np.array_equal(np.sort(g[i].ravel()), np.sort(f[i].ravel()))


def test_rest_state_is_fixed_point():
    for periodic in [(False,) * 3, (True, False, True), (True,) * 3]:
        f = lbm.rest_state((6, 5, 4))
        g = lbm.step_bulk(f, TAU, periodic=periodic)
        assert np.allclose(g, f, atol=1e-16)


def test_closed_box_conserves_mass():
    f = _random_state((6, 7, 8), seed=4)
    m0 = f.sum()
    for _ in range(30):
        f = lbm.step_bulk(f, TAU, periodic=(False, False, False))
    assert abs(f.sum() - m0) / m0 < 1e-13


def test_wall_momentum_balance_moving_lid():
    # From rest, a lid (y+ wall) moving at U adds to every population it
    # reflects the moving-wall term 6 w_i rho0 (e_i.U); collision conserves
    # momentum, so the x-momentum after one step is the sum of e_ix times that
    # term over the reflected directions (e_iy = -1) and the lid nodes.
    shape = (3, 6, 4)
    f = lbm.rest_state(shape)
    wv = np.zeros((6, 3))
    wv[3] = (0.01, 0, 0)
    g = lbm.step_bulk(f, TAU, periodic=(True, False, True), wall_velocity=wv)
    mx = np.einsum("i,i...->...", E[:, 0].astype(float), g).sum()
    expect = 0.0
    for i in range(Q):
        if E[i, 1] == -1:
            expect += 6 * W[i] * E[i, 0] * 0.01 * E[i, 0]
    expect *= shape[0] * shape[2]
    assert abs(mx - expect) < 1e-15


def test_couette_linear_profile():
    # Plane Couette flow, lid (y+ wall) moving at U along x: the steady profile
    # is exactly linear, u_x(y) = U (y + 1/2) / H with walls at -1/2, H - 1/2.
    H, U = 8, 0.01
    wv = np.zeros((6, 3))
    wv[3] = (U, 0, 0)
    f = lbm.rest_state((1, H, 1))
    for _ in range(4000):
        f = lbm.step_bulk(f, TAU, periodic=(True, False, True), wall_velocity=wv)
    rho, u = lbm.moments(f)
    y = np.arange(H)
    assert np.max(np.abs(u[0, 0, :, 0] - U * (y + 0.5) / H)) < 1e-8 * U
    assert np.max(np.abs(u[1:])) < 1e-14
    assert np.max(np.abs(rho - 1.0)) < 1e-12


@pytest.mark.parametrize("H", [16, 32])
def test_poiseuille_closed_form(H):
    # Body-force driven channel: u(y) = g (y + 1/2)(H - 1/2 - y) / (2 nu),
    # nu = (tau - 1/2)/3.  The discrete solution has exactly the closed-form
    # curvature u'' = -g/nu; halfway bounce-back adds a uniform slip whose
    # size relative to u_max decays like H^-2.
    g = 1e-6
    nu = (TAU - 0.5) / 3.0
    y = np.arange(H)
    ua = g / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    u0 = np.zeros((3, 1, H, 1))
    u0[0, 0, :, 0] = ua
    f = lbm.equilibrium(np.ones((1, H, 1)), u0)
    for _ in range(5000 if H == 16 else 12000):
        f = lbm.step_bulk(f, TAU, periodic=(True, False, True), force=(g, 0, 0))
    _, u = lbm.moments(f, force=(g, 0, 0))
    un = u[0, 0, :, 0]
    curv = np.diff(un, 2)
    assert np.allclose(curv, -g / nu, rtol=1e-7)
    slip = un - ua
    assert np.max(np.abs(slip - slip.mean())) < 1e-6 * ua.max()
    assert abs(slip.mean()) / ua.max() < 1.2 * (16.0 / H) ** 2 * 1.1e-3


def test_update_cells_matches_full_step():
    shape = (5, 6, 7)
    f = _random_state(shape, seed=5)
    wv = np.zeros((6, 3))
    wv[1] = (0, 0.02, -0.01)
    for periodic in [(False, False, False), (True, False, True)]:
        full = lbm.step_bulk(f, TAU, periodic=periodic, wall_velocity=wv)
        cells = np.array(list(itertools.product(range(7), range(6), range(5))))
        part = lbm.update_cells(f, cells, TAU, periodic=periodic, wall_velocity=wv)
        ref = full[:, cells[:, 2], cells[:, 1], cells[:, 0]]
        assert np.allclose(part, ref, atol=1e-16)
