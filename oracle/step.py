"""The whole coupled step of the oracle (test infrastructure only): flag at the
current pose, the coupled LBM step (refill, stream with bounce-back, collide,
momentum exchange), then dem_substeps DEM substeps of contact forces and
rigid-body update with the hydrodynamic force held fixed (reading A13; the
paper runs 100 DEM substeps per LBM step, Sec. 3)."""
import numpy as np

from . import contact, coupling, dem, metaball


class OracleState:
    """Populations, particle states, previous owners and contact springs."""

    def __init__(self, shape, f, particles, tau=0.8, periodic=(False, False, False), wall_velocity=None,
                 gravity=(0.0, 0.0, 0.0), rho0=1.0, bb_mode="ibb", dem_substeps=1, contact_params=None,
                 cover_uncover=False):
        self.shape = tuple(shape)
        self.f = np.asarray(f, dtype=np.float64)
        self.particles = [dict(P) for P in particles]
        self.tau = tau
        self.periodic = tuple(periodic)
        self.wall_velocity = wall_velocity
        self.gravity = gravity
        self.rho0 = rho0
        self.bb_mode = bb_mode
        self.dem_substeps = dem_substeps
        self.cover_uncover = cover_uncover   # reading A11's option (coupling.coupled_lbm_step)
        self.contact_params = contact_params or {"kn": 1.0, "kt": 2.0 / 7.0, "eta_n": 0.0, "eta_t": 0.0,
                                                 "mu_s": 0.4}
        self.owner_prev = np.full((shape[2], shape[1], shape[0]), -1, dtype=np.int64)
        if cover_uncover:
            # the particles are not inserted into the fluid: the first step
            # covers nothing (without the option the two starts are the same)
            self.owner_prev = metaball.flag_nodes(self.shape, self.particles)
        self.history = {}
        self.F_hydro = np.zeros((len(particles), 3))
        self.T_hydro = np.zeros((len(particles), 3))
        self.F_contact = np.zeros((len(particles), 3))
        self.T_contact = np.zeros((len(particles), 3))
        self.contacts = []


def step(S):
    """Advance the oracle state by one coupled step (in place)."""
    owner = metaball.flag_nodes(S.shape, S.particles)
    S.f, S.F_hydro, S.T_hydro = coupling.coupled_lbm_step(
        S.f, owner, S.owner_prev, S.particles, S.tau, bb_mode=S.bb_mode, periodic=S.periodic,
        wall_velocity=S.wall_velocity, rho0=S.rho0, cover_uncover=S.cover_uncover)
    S.owner_prev = owner
    dt = 1.0 / S.dem_substeps
    for _ in range(S.dem_substeps):
        Fc, Tc, S.history, S.contacts = contact.contact_forces(S.particles, S.shape, S.periodic, S.contact_params,
                                                               S.history, dt)
        S.F_contact, S.T_contact = Fc, Tc
        S.particles = [dem.integrate(P, S.F_hydro[i] + Fc[i], S.T_hydro[i] + Tc[i], S.gravity, S.rho0, dt)
                       for i, P in enumerate(S.particles)]
    return S
