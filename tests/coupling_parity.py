"""Shared parts of the GPU parity tests of one coupled LBM step (flagging,
links, refill, IBB, momentum exchange) against the FP64 oracle: particle
preparation, seeded initial flows, the one-step GPU run through the C-ABI and
the element-wise comparison.  Test plumbing only.

Bars (north star and the parity protocol of the scope table): node owners,
node classes and the link set bit-exact; wall fraction q within 1e-5;
populations at fluid nodes within 1e-5 relative; hydrodynamic force and torque
within 1e-4 * max(|F_ref|, 1e-3 * sum_links |dP|) per particle (the link-sum
scale guards the cancellation of O(0.1) link terms into a small net force).
"""
import numpy as np

from oracle import coupling, lbm, metaball
from oracle.d3q19 import E
from paper_2209_10411_gb300 import scenes

TAU = 0.8
ALL_LBM = 1 | 2 | 4 | 8 | 16 | 32  # flag, links, refill, bulk, boundary, swap
Q_TOL = 1e-5
POP_TOL = 1e-5
FT_TOL = 1e-4


def prepared(spec, pos, quat, vel, omega):
    """Oracle particle dict with control points shifted to the oracle's
    quadrature centroid (inputs to both sides)."""
    mp = metaball.mass_properties(spec.centers, spec.k, spec.density)
    c = spec.centers - mp["centroid"]
    mp = metaball.mass_properties(c, spec.k, spec.density)
    return {"centers": c, "k": spec.k.copy(), "pos": np.asarray(pos, float), "quat": np.asarray(quat, float),
            "vel": np.asarray(vel, float), "omega": np.asarray(omega, float), "density": spec.density,
            "skin": spec.skin, "mass": mp["mass"], "volume": mp["volume"], "inertia": mp["inertia"]}


def initial_flow(shape, seed, umax=0.03):
    """f = f^eq(1, u) (1 + 0.01 xi) with a smooth random u of amplitude umax,
    rounded to float32 (both sides read the same bits)."""
    nx, ny, nz = shape
    u = umax * scenes.velocity_field_noise(shape, seed)
    feq = lbm.equilibrium(np.ones((nz, ny, nx)), u)
    noise = scenes.lattice_noise(shape, seed).astype(np.float64)
    return (feq * (1.0 + 0.01 * noise)).astype(np.float32).astype(np.float64)


def add_particles(sim, parts):
    for P in parts:
        sim.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})


def run_one_step(B, shape, parts_prev, parts, f0, mode, storage=0, phases=ALL_LBM, cover_uncover=False,
                 max_particles=None):
    """GPU: flag at the previous poses, then one step of the given phases at
    the current poses from the populations f0 (handle capacity max_particles,
    by default the particle count, at least 4)."""
    nx, ny, nz = shape
    sim = B.Simulation(nx, ny, nz, tau=TAU, bb_mode=(B.BB_LADD if mode == "ladd" else B.BB_IBB), storage=storage,
                       max_particles=max_particles or max(4, len(parts)))
    add_particles(sim, parts_prev)
    sim.step_phases(1)  # flags at the previous pose
    if cover_uncover:
        sim.set_momentum_rules(cover_uncover=True)
    for i, P in enumerate(parts):
        sim.set_particle_state(i, P["pos"], P["quat"], P["vel"], P["omega"])
    sim.set_populations(f0.astype(np.float32))
    sim.step_phases(phases)
    return sim


def compare_step(sim, shape, parts_prev, parts, f0, mode):
    """Element-wise comparison of the GPU's step with the oracle's.  Asserts
    the bars and returns the measured errors (max |dq|, max relative
    population error, per-particle force and torque errors over their
    scales) and the counts that were compared."""
    nx, ny, nz = shape
    owner = metaball.flag_nodes(shape, parts)
    owner_prev = metaball.flag_nodes(shape, parts_prev)
    ref, F, T, L = coupling.coupled_lbm_step(f0, owner, owner_prev, parts, TAU, bb_mode=mode, return_links=True)
    cls, own = sim.node_classes()
    own = own.astype(np.int64)
    own[own == 0xFFFFFFFF] = -1
    # owners and classes bit-exact
    assert np.array_equal(own, owner), "owner mismatch at %d nodes" % (own != owner).sum()
    solid, new = coupling.classify(owner, owner_prev)
    boundary = np.zeros_like(solid)
    cl = L["cell"]
    boundary[cl[:, 2], cl[:, 1], cl[:, 0]] = True
    assert np.array_equal((cls & 1) != 0, solid)
    assert np.array_equal((cls & 2) != 0, boundary)
    assert np.array_equal((cls & 4) != 0, new)
    # link set bit-exact, q within Q_TOL
    g = sim.links()
    lin_ref = (cl[:, 2] * ny + cl[:, 1]) * nx + cl[:, 0]
    key_ref = np.stack([L["particle"], lin_ref, L["dir"]], 1)
    key_gpu = np.stack([g["particle"].astype(np.int64), g["cell"].astype(np.int64), g["dir"].astype(np.int64)], 1)
    o_ref = np.lexsort(key_ref.T[::-1])
    o_gpu = np.lexsort(key_gpu.T[::-1])
    assert np.array_equal(key_ref[o_ref], key_gpu[o_gpu]), "link sets differ (%d vs %d links)" % (
        len(key_ref), len(key_gpu))
    dq = np.abs(g["q"][o_gpu].astype(np.float64) - L["q"][o_ref])
    dq_max = float(dq.max()) if len(dq) else 0.0
    assert dq_max < Q_TOL, "max |dq| %g" % dq_max
    # populations at fluid nodes
    got = sim.get_populations().astype(np.float64)
    fl = owner < 0
    rel = np.abs(got[:, fl] - ref[:, fl]) / np.abs(ref[:, fl])
    pop_max = float(rel.max())
    assert pop_max < POP_TOL, "max rel population err %g" % pop_max
    # force and torque
    fr = sim.forces()
    dP = L["dP"]
    errF, errT = [], []
    for p in range(len(parts)):
        m = L["particle"] == p
        if not m.any():
            continue
        qw = np.full(m.sum(), 0.5) if mode == "ladd" else L["q"][m]
        xw = L["cell"][m] + qw[:, None] * E[L["dir"][m]]
        arm = xw - parts[p]["pos"]
        scaleF = max(np.linalg.norm(F[p]), 1e-3 * np.abs(dP[m]).sum())
        scaleT = max(np.linalg.norm(T[p]), 1e-3 * np.abs(np.cross(arm, dP[m])).sum())
        eF = np.linalg.norm(fr["F_hydro"][p] - F[p]) / scaleF
        eT = np.linalg.norm(fr["T_hydro"][p] - T[p]) / scaleT
        errF.append(float(eF))
        errT.append(float(eT))
        assert eF <= FT_TOL, ("force", p, fr["F_hydro"][p], F[p], eF)
        assert eT <= FT_TOL, ("torque", p, fr["T_hydro"][p], T[p], eT)
    return {"F": F, "T": T, "dq_max": dq_max, "pop_rel_max": pop_max, "force_err": errF, "torque_err": errT,
            "links": int(len(key_ref)), "boundary_nodes": int(boundary.sum()), "solid_nodes": int(solid.sum()),
            "new_nodes": int(new.sum())}
