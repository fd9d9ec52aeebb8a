"""Benchmark of the MI-DELBM coupled step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                    [--config c2] [--storage f32|f16|bf16]

A step is one pass of the whole per-timestep path (flagging, links, refill,
bulk stream-collide, boundary IBB + momentum exchange, contacts, rigid-body
update) over the synthetic settling tank.  Default workload: 256x256x512
lattice, three cobblestone-like particles of 24-40 metaballs, FP32 storage.

Prints one JSON line (rank 0).  value = whole-job MLUPS (lattice nodes times
steps over the device-timed region, summed over ranks; each rank runs its own
independent tank, so scaling is weak and no data-path collective exists).
--impl reference times the FP64 oracle on this machine's host cores on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE = {0: 152, 1: 76, 2: 76}   # 19 loads + 19 stores of the stored type
# DRAM bytes (read + write) of one bulk launch on the 256x256x512 tank, from
# ncu captures of the same kernels on 256x256x128 scaled by the nodes
# processed (profiles/k_bulk_stream_collide_f32.md, k_bulk_quad16_f16.md);
# keyed by (storage, four-node kernel).  Reported only for the kernel that
# was captured.
BULK_TRAFFIC = {(0, False): 4 * 1222.0e6, (1, True): 4 * 591.1e6}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
DTYPE_NAME = {0: "f32", 1: "f16-dev/f32-compute", 2: "bf16-dev/f32-compute"}
def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=None):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_index is not None:
            cmd[1:1] = ["-i", str(self.gpu_index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU side: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def cores_used(cpu_s, wall_s):
    """Threads a timed CPU region kept busy: process CPU time (all threads)
    over wall time, at least 1."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


_TANK_FRACTION = {}


def tank_boundary_fraction(seed=0):
    """Boundary nodes (fluid nodes with a link into a particle) per lattice
    node of the settling tank, from the oracle's flags of each cobble alone."""
    if seed not in _TANK_FRACTION:
        from oracle import coupling, metaball
        from paper_2209_10411_gb300 import scenes
        scene = scenes.config2(seed=seed)
        nb = 0
        for spec in scene.particles:
            side = int(np.ceil(2.0 * metaball.bounding_radius(spec.centers, spec.k))) + 4
            P = {"centers": spec.centers, "k": spec.k, "pos": np.array([side / 2.0] * 3), "quat": spec.quat}
            cell, _, _ = coupling.find_links(metaball.flag_nodes((side, side, side), [P]))
            nb += len(np.unique(cell, axis=0))
        _TANK_FRACTION[seed] = nb / float(np.prod(scene.shape))
    return _TANK_FRACTION[seed]


class OracleSample:
    """A bounded sample of the tank's coupled step for the oracle: a crop^3
    window with the same share of boundary nodes as the whole tank, made by
    placing the first cobble beside the window so that a cap of its surface
    reaches in (gravity runs along the window face, so the cap keeps its size
    while the cobble settles).  Each step is the oracle's coupled LBM step
    (flags, links, refill, IBB, momentum exchange, stream-collide) plus the
    rigid-body update; the window is set up once and run() continues it."""

    def __init__(self, crop=96, seed=0):
        from oracle import coupling, dem, lbm, metaball
        from paper_2209_10411_gb300 import scenes
        self.mods = (coupling, dem, metaball)
        scene = scenes.config2(seed=seed)
        spec = scene.particles[0]
        self.crop = crop
        self.shape = (crop, crop, crop)
        self.gravity = tuple(float(g) for g in scene.gravity)
        # the cobble's own mass properties (unit-spacing quadrature), control
        # points about its centroid
        mp = metaball.mass_properties(spec.centers, spec.k, spec.density, h=1.0)
        P = {"centers": spec.centers - mp["centroid"], "k": spec.k, "quat": spec.quat, "vel": np.zeros(3),
             "omega": np.zeros(3), "mass": mp["mass"], "volume": mp["volume"], "inertia": mp["inertia"]}
        self.target = max(1, int(round(tank_boundary_fraction(seed) * crop ** 3)))

        def boundary_nodes(depth):
            P["pos"] = np.array([-depth, crop / 2.0, crop / 2.0 + 0.37])
            owner = metaball.flag_nodes(self.shape, [P])
            xs = np.nonzero((owner >= 0).any(axis=(0, 1)))[0]
            if len(xs) == 0:
                return 0
            # boundary nodes lie within one node of the solid: count on the slab
            cell, _, _ = coupling.find_links(owner[:, :, :min(crop, int(xs.max()) + 3)])
            return len(np.unique(cell, axis=0))

        lo, hi = 0.0, metaball.bounding_radius(P["centers"], P["k"])   # cap largest at lo, empty at hi
        for _ in range(16):
            mid = 0.5 * (lo + hi)
            if boundary_nodes(mid) > self.target:
                lo = mid
            else:
                hi = mid
        self.boundary = boundary_nodes(lo)
        self.P = P
        self.f = lbm.rest_state(self.shape)
        self.owner_prev = metaball.flag_nodes(self.shape, [self.P])

    def step(self):
        coupling, dem, metaball = self.mods
        owner = metaball.flag_nodes(self.shape, [self.P])
        self.f, F, T = coupling.coupled_lbm_step(self.f, owner, self.owner_prev, [self.P], 0.8)
        self.P = dem.integrate(self.P, F[0], T[0], self.gravity)
        self.owner_prev = owner

    def run(self, budget_s=0.0):
        """One step or more, until about budget_s seconds of CPU work;
        returns (MLUPS, seconds, steps)."""
        t0 = time.perf_counter()
        c0 = time.process_time()
        steps = 0
        while True:
            self.step()
            steps += 1
            dt = time.perf_counter() - t0
            if dt >= budget_s:
                break
        self.cores = cores_used(time.process_time() - c0, dt)
        return self.crop ** 3 * steps / dt / 1e6, dt, steps

    def describe(self):
        return ("FP64 numpy oracle: coupled step + rigid-body update on a %d^3 window holding a cap of one "
                "cobble with %d boundary nodes, the tank's share (%.2e per node)"
                % (self.crop, self.boundary, tank_boundary_fraction()))


def _oracle_worker(crop, budget_s, warmup_steps, timed_steps, barrier, queue):
    """One host core's share of the all-core oracle timing (a spawned process:
    it never touches the GPU): its own window of the tank, warm-up steps, then
    after the barrier either timed_steps steps or steps until budget_s."""
    try:
        sampler = OracleSample(crop=crop)
        sampler.run()                          # the first step pays numpy's one-time costs
        for _ in range(warmup_steps):
            sampler.run()
        barrier.wait()
        t0 = time.time()
        steps = 0
        if timed_steps:
            for _ in range(timed_steps):
                sampler.run()
            steps = timed_steps
        else:
            _, _, steps = sampler.run(budget_s=budget_s)
        queue.put((steps, t0, time.time(), None))
    except Exception as e:  # reported by the parent
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put((0, 0.0, 0.0, repr(e)))


def oracle_all_cores(crop, budget_s=15.0, warmup_steps=0, timed_steps=0, n=None):
    """The oracle on every host core at once: n = os.cpu_count() spawned
    processes, each on its own crop^3 window, released together by a barrier.
    Returns (whole-box MLUPS over the span from the first start to the last
    end, that span in s, the steps of each process, n)."""
    import multiprocessing as mp
    n = n or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n)
    queue = ctx.Queue()
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"                    # one thread per process: n processes on n cores
    procs = [ctx.Process(target=_oracle_worker, args=(crop, budget_s, warmup_steps, timed_steps, barrier, queue))
             for _ in range(n)]
    try:
        for p_ in procs:
            p_.start()
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res = [queue.get(timeout=900) for _ in range(n)]
    for p_ in procs:
        p_.join(timeout=60)
    errs = [r[3] for r in res if r[3]]
    if errs:
        raise RuntimeError("oracle worker failed: " + errs[0])
    span = max(r[2] for r in res) - min(r[1] for r in res)
    steps = [r[0] for r in res]
    return crop ** 3 * sum(steps) / span / 1e6, span, steps, n


def c2_window_parity(B, sim, scene, crop=96):
    """The settling tank's force and torque against the FP64 oracle on a
    cropped copy: the crop^3 window around the first cobble, holding the
    tank's populations and every particle that reaches into it, with the
    poses of the tank's last two steps (flags at the earlier one), one
    coupled LBM step on both sides (the window's faces are closed walls on
    both).  Bar: |F - F_ref| <= 1e-4 max(|F_ref|, 1e-3 sum_links |dP|) per
    particle, likewise the torque."""
    import torch
    from oracle import coupling, metaball
    from oracle.d3q19 import E
    nx, ny, nz = scene.shape
    npart = sim.num_particles()
    prev = [sim.get_particle_state(i) for i in range(npart)]
    sim.step(1)
    sim.synchronize()
    cur = [sim.get_particle_state(i) for i in range(npart)]
    shapes = [sim.get_particle_shape(i) for i in range(npart)]
    lo = [int(min(max(round(cur[0]["pos"][a]) - crop // 2, 0), n - crop)) for a, n in enumerate((nx, ny, nz))]
    v = sim.device_view()
    assert v.storage == B.STORE_F32
    pop = torch.as_tensor(B.CudaArray(v.populations, (19, v.plane_stride), "<f4"), device="cuda")
    r = [torch.arange(lo[a], lo[a] + crop, device="cuda", dtype=torch.int64) for a in range(3)]
    zz, yy, xx = torch.meshgrid(r[2], r[1], r[0], indexing="ij")
    lin = ((zz * ny + yy) * nx + xx).reshape(-1)
    f0 = pop.index_select(1, lin).cpu().numpy().astype(np.float64).reshape(19, crop, crop, crop)
    shift = np.array(lo, dtype=float)
    parts, parts_prev, ids = [], [], []
    for i in range(npart):
        X = cur[i]["pos"] - shift
        if np.any(X + shapes[i]["Rb"] < -1) or np.any(X - shapes[i]["Rb"] > crop):
            continue
        base = {"centers": shapes[i]["centers"], "k": shapes[i]["k"], "mass": shapes[i]["mass"],
                "volume": shapes[i]["volume"], "inertia": shapes[i]["inertia"], "density": scene.particles[i].density,
                "skin": scene.particles[i].skin}
        parts.append(dict(base, pos=X, quat=cur[i]["quat"], vel=cur[i]["vel"], omega=cur[i]["omega"]))
        parts_prev.append(dict(base, pos=prev[i]["pos"] - shift, quat=prev[i]["quat"], vel=prev[i]["vel"],
                               omega=prev[i]["omega"]))
        ids.append(i)
    shape = (crop, crop, crop)
    win = B.Simulation(crop, crop, crop, tau=scene.tau, storage=B.STORE_F32, max_particles=max(4, len(parts)))
    for P in parts_prev:
        win.add_particle(P["centers"], P["k"], P["density"], P["skin"], P["pos"], P["quat"], P["vel"], P["omega"],
                         mass_props={"mass": P["mass"], "volume": P["volume"], "inertia": P["inertia"]})
    win.step_phases(B.PHASE_FLAG)
    for j, P in enumerate(parts):
        win.set_particle_state(j, P["pos"], P["quat"], P["vel"], P["omega"])
    win.set_populations(f0.astype(np.float32))
    win.step_phases(B.PHASE_FLAG | B.PHASE_LINKS | B.PHASE_REFILL | B.PHASE_BULK | B.PHASE_BOUNDARY | B.PHASE_SWAP)
    fr = win.forces()
    gl = win.links()
    win.close()
    t0 = time.perf_counter()
    owner = metaball.flag_nodes(shape, parts)
    owner_prev = metaball.flag_nodes(shape, parts_prev)
    _, F, T, L = coupling.coupled_lbm_step(f0, owner, owner_prev, parts, scene.tau, return_links=True)
    oracle_s = time.perf_counter() - t0
    per = []
    for j, i in enumerate(ids):
        m = L["particle"] == j
        if not m.any():
            continue   # reaches into the window's box but not its nodes
        arm = L["cell"][m] + L["q"][m][:, None] * E[L["dir"][m]] - parts[j]["pos"]
        sF = max(np.linalg.norm(F[j]), 1e-3 * np.abs(L["dP"][m]).sum())
        sT = max(np.linalg.norm(T[j]), 1e-3 * np.abs(np.cross(arm, L["dP"][m])).sum())
        per.append({"particle": i, "links": int(m.sum()),
                    "force_err": float(np.linalg.norm(fr["F_hydro"][j] - F[j]) / sF),
                    "torque_err": float(np.linalg.norm(fr["T_hydro"][j] - T[j]) / sT),
                    "F_ref": [float(x) for x in F[j]]})
    return {"window": [crop] * 3, "corner": lo, "links_oracle": int(len(L["dir"])), "links_gpu": int(len(gl["dir"])),
            "force_err_max": max(p_["force_err"] for p_ in per), "torque_err_max": max(p_["torque_err"] for p_ in per),
            "bar": 1e-4, "particles": per, "oracle_s": oracle_s,
            "scale": "max(|F_ref|, 1e-3 sum_links |dP|) per particle (torque likewise)"}


def cpu_leg(B, sim, scene, budget_s):
    """The oracle beside the GPU (rank 0, one GPU): the tank's cropped-copy
    force/torque error, then the oracle's throughput on one host core and on
    all of them (the window with the tank's share of boundary nodes)."""
    out = {}
    try:
        out["c2_force_error"] = c2_window_parity(B, sim, scene)
    except Exception as e:
        out["c2_force_error"] = {"error": repr(e)}
    sampler = OracleSample(crop=96)
    v1, dt, n = sampler.run(budget_s=budget_s)
    single = {"value": v1, "unit": "MLUPS", "cores": sampler.cores, "steps": n, "s": dt}
    try:
        vall, span, steps, ncores = oracle_all_cores(96, budget_s=budget_s)
        cpu = {"value": vall, "unit": "MLUPS", "cores": ncores, "kind": "oracle",
               "sample": sampler.describe() + "; %d processes (one per host core), each its own window, %d steps "
                         "in %.1f s in total" % (ncores, sum(steps), span),
               "single_core": single}
    except Exception as e:
        cpu = dict(single, kind="oracle", sample=sampler.describe() + ", %d steps in %.1f s (all-core run failed: %r)"
                   % (n, dt, e))
    out["cpu_baseline"] = cpu
    return out


def run_reference(args):
    """The oracle on all host cores: one process per core, each of the K timed
    steps one oracle step per process on its own window of the tank with the
    tank's share of boundary nodes, the window's edge sized from a one-core
    calibration so that the whole warm-up + timed run takes about REF_TOTAL_S
    seconds (between 24 and 96 nodes); value = all processes' node updates
    over the span from the first start to the last end."""
    from paper_2209_10411_gb300 import replicas
    rank, world, _ = replicas.rank_env()
    if rank != 0:
        return
    nsteps = max(1, args.steps + args.warmup)
    per_step = min(60.0, REF_TOTAL_S / nsteps)
    cal = OracleSample(crop=32)
    cal.run()                      # first step pays numpy's one-time costs
    _, dt, n = cal.run(budget_s=0.5)
    t_node = dt / n / 32 ** 3
    crop = int(max(24, min(96, (per_step / t_node) ** (1.0 / 3.0))))
    value, span, steps, ncores = oracle_all_cores(crop, warmup_steps=args.warmup, timed_steps=args.steps)
    sampler = OracleSample(crop=crop)
    sample = (sampler.describe() + "; %d processes (one per host core), each its own window, %d timed steps each "
              "after %d warm-up steps" % (ncores, args.steps, args.warmup))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": span / max(1, args.steps) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": CONFIG,
           "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": ncores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


REF_TOTAL_S = 100.0  # the reference arm's warm-up + timed steps, about (per process, all cores busy)


METRIC = "coupled-step MLUPS (FP32 vs FP16-store) at stated err; contact solves/s"
CONFIG = {}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
SCHEDULE = {"overlap": False}   # --schedule: boundary nodes beside the bulk kernel


def build_sim(B, scene, storage, stream, dem_substeps=1):
    nx, ny, nz = scene.shape
    sim = B.Simulation(nx, ny, nz, tau=scene.tau, gravity=scene.gravity, storage=storage, stream=stream,
                       max_particles=max(16, len(scene.particles)),
                       max_balls=max(65536, sum(len(p.k) for p in scene.particles)), dem_substeps=dem_substeps)
    for p in scene.particles:
        sim.add_particle(p.centers, p.k, p.density, p.skin, p.pos, p.quat, p.vel, p.omega)
    if SCHEDULE["overlap"]:
        sim.set_schedule(overlap_boundary=True)
    return sim


def train_guess(B):
    """The learned Newton guess: 2M pair solves of 256 bed shapes (seed 1,
    shapes and poses independent of the timed bed) made by the plain Newton
    kernel, and 12k AdamW steps of the BF16 network on them (library
    kernels; not timed)."""
    import torch
    from paper_2209_10411_gb300 import guess
    t0 = time.perf_counter()
    shapes = guess.bed_shapes(1, 256)
    sim = B.Simulation(16, 16, 16, max_particles=len(shapes) + 1, max_balls=sum(len(s["k"]) for s in shapes) + 1)
    guess.add_shapes(sim, shapes)
    # centre distances of the bed's candidates: 0.5 to 1.6 times R_i + R_j
    ij, poses = guess.pair_poses(1, shapes, 2_000_000, spacing=(0.5, 1.5))
    X, T, _ = guess.generate(sim, *guess.to_device(ij, poses))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    params, hist = guess.train(X, T, steps=12000, batch=4096, lr=2e-3, seed=0, log_every=4000, standardize=True,
                               target_weights=(10.0, 10.0, 10.0, 1.0))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    sim.close()
    info = {"solves": 2_000_000, "samples": int(X.shape[0]), "steps": 12000, "batch": 4096,
            "generate_s": t1 - t0, "train_s": t2 - t1, "loss": hist}
    return params, info


CONTACT_FLOP_PER_BALL_ITER = 35   # x - c, r^2, 1/r^2, k/r^2, gradient, six Hessian entries
CONTACT_FLOP_SOLVE = 60           # the 3x3 (pairs) solve per iteration
CONTACT_FLOP_SOLVE_WALL = 100     # the 4x4 (walls) solve per iteration


def contact_flops(recs, nballs):
    """Algorithmic FLOPs of the Newton iterations of these contact records:
    per iteration 35 per ball of both particles plus the 3x3 solve (pairs), or
    35 per ball plus the 4x4 solve (walls).  The plain start's sphere-gap
    search and the contact forces are not counted."""
    total = 0.0
    for c in recs:
        if c["j"] >= 0:
            total += c["iters"] * (CONTACT_FLOP_PER_BALL_ITER * (nballs[c["i"]] + nballs[c["j"]]) + CONTACT_FLOP_SOLVE)
        else:
            total += c["iters"] * (CONTACT_FLOP_PER_BALL_ITER * nballs[c["i"]] + CONTACT_FLOP_SOLVE_WALL)
    return total


def contact_solves(B, scenes, args, alu=None):
    """Contact solves per second: the DEM contact phase alone (broad phase +
    persistent Newton/force kernel; with the learned guess also the feature
    kernel and the MLP) on the 3000-particle bed of 4-128 balls in
    384x384x768, timed with CUDA events over repeated substeps, with the
    plain guess and with the learned guess."""
    sc = scenes.config5()
    nx, ny, nz = sc.shape
    periodic = (False, False, False)
    if args.small_contact_lattice:  # profiling case: the same particles and pairs, no lattice memory, no walls
        nx, ny, nz = 16, 16, 16
        periodic = (True, True, True)
    params, train_info = train_guess(B)
    out = {}
    recs_by_mode = {}
    for mode in ("plain", "learned"):
        sim = B.Simulation(nx, ny, nz, tau=sc.tau, storage=1, max_particles=len(sc.particles),
                           max_balls=sum(len(p.k) for p in sc.particles) + 16, kn=1.0, kt=2.0 / 7.0,
                           periodic=periodic)
        for p in sc.particles:
            r = p.nominal_radius
            vol = 4.0 / 3.0 * np.pi * r ** 3
            m = p.density * vol
            sim.add_particle(p.centers, p.k, p.density, p.skin, p.pos, p.quat,
                             mass_props={"mass": m, "volume": vol, "inertia": np.eye(3) * 0.4 * m * r * r})
        if mode == "learned":
            sim.set_guess(B.GUESS_LEARNED, params)
        sim.set_timing(True)
        for _ in range(3):
            sim.step_phases(B.PHASE_CONTACT)
        sim.phase_times(reset=True)
        reps = 20
        for _ in range(reps):
            sim.step_phases(B.PHASE_CONTACT)
        kc = sim.kernel_time("k_contacts")
        pt = sim.phase_times(reset=True)["contact"]
        recs = sim.contacts()
        sim.close()
        recs_by_mode[mode] = recs
        kc_ms = kc[0] / max(kc[1], 1)
        n = len(recs)
        pair_iters = np.array([c["iters"] for c in recs if c["j"] >= 0])
        status = np.bincount(np.array([c["status"] for c in recs], dtype=int), minlength=5)
        ms = pt[0] / reps
        out[mode] = {"value": n / (ms * 1e-3), "unit": "solves/s", "candidates": n,
                     "pairs": int(len(pair_iters)),
                     "in_contact": int(sum(1 for c in recs if c["delta"] > 0 and c["status"] == 0)),
                     "mean_pair_iters": float(pair_iters.mean()) if len(pair_iters) else None,
                     "status_counts": {"ok": int(status[0]), "not_converged": int(status[1]),
                                       "singular": int(status[2]), "inside_core": int(status[3]),
                                       "out_of_range": int(status[4])},
                     "ms_per_substep": ms, "launches_per_substep": pt[1] / reps,
                     "k_contacts_ms": kc_ms}
        if alu:
            fl = contact_flops(recs, [len(p.k) for p in sc.particles])
            tf = fl / (kc_ms * 1e-3) / 1e12
            out[mode]["roofline"] = {"bound": "alu", "kernel": "k_contacts (Newton closest points and forces)",
                                     "achieved": tf, "peak": alu["fp32_tflops"], "unit": "TFLOP/s",
                                     "frac": tf / alu["fp32_tflops"], "peak_kind": "measured (mi_measure_fma_peak)",
                                     "algorithmic_flop_per_launch": fl,
                                     "flop_per_iteration": "35 (n_i + n_j) + 60 per pair, 35 n_i + 100 per wall",
                                     "traffic": None}
    # DEM substeps of a moving bed (contact + rigid-body update, 10 substeps per
    # call: the particles move between substeps), plain vs warm start
    moving = {}
    for name, mode in (("plain", B.GUESS_PLAIN), ("warm", B.GUESS_WARM)):
        sim = B.Simulation(nx, ny, nz, tau=sc.tau, storage=1, max_particles=len(sc.particles),
                           max_balls=sum(len(p.k) for p in sc.particles) + 16, kn=1.0, kt=2.0 / 7.0,
                           periodic=periodic, dem_substeps=10, guess_mode=mode, gravity=sc.gravity)
        for p in sc.particles:
            r = p.nominal_radius
            vol = 4.0 / 3.0 * np.pi * r ** 3
            m = p.density * vol
            sim.add_particle(p.centers, p.k, p.density, p.skin, p.pos, p.quat,
                             mass_props={"mass": m, "volume": vol, "inertia": np.eye(3) * 0.4 * m * r * r})
        sim.set_timing(True)
        for _ in range(2):
            sim.step_phases(B.PHASE_CONTACT | B.PHASE_INTEGRATE)
        sim.phase_times(reset=True)
        calls = 3
        for _ in range(calls):
            sim.step_phases(B.PHASE_CONTACT | B.PHASE_INTEGRATE)
        pt = sim.phase_times(reset=True)
        recs = sim.contacts()
        sim.close()
        it = np.array([c["iters"] for c in recs if c["j"] >= 0 and c["status"] == 0])
        ms = pt["contact"][0] / (10 * calls)
        moving[name] = {"value": len(recs) / (ms * 1e-3), "unit": "solves/s", "ms_per_substep": ms,
                        "mean_pair_iters_last_substep": float(it.mean()) if len(it) else None,
                        "candidates": len(recs)}
    # the two modes must agree: same converged pairs, same contact points (1e-5 of 2 R_b)
    rb = {i: None for i in range(len(sc.particles))}
    for i, p in enumerate(sc.particles):
        rb[i] = float(np.sqrt((p.centers ** 2).sum(1)).max() + np.sqrt(p.k.sum()))
    a = {(c["i"], c["j"]): c for c in recs_by_mode["plain"] if c["j"] >= 0 and c["status"] == 0}
    b = {(c["i"], c["j"]): c for c in recs_by_mode["learned"] if c["j"] >= 0 and c["status"] == 0}
    same = [np.linalg.norm(a[k]["x_cp"] - b[k]["x_cp"]) <= 2e-5 * max(rb[k[0]], rb[k[1]]) for k in a if k in b]
    res = dict(out["plain"])
    wl = sc.name + (" (16^3 periodic lattice: profiling case, no walls)" if args.small_contact_lattice else "")
    res.update({"guess": "plain", "workload": wl, "particles": len(sc.particles), "learned": out["learned"],
                "learned_vs_plain": {"solves_per_s": out["learned"]["value"] / out["plain"]["value"],
                                     "pair_iters": (out["learned"]["mean_pair_iters"] or 0) /
                                     max(out["plain"]["mean_pair_iters"] or 1, 1e-9),
                                     "converged_pairs_plain": len(a), "converged_pairs_learned": len(b),
                                     "same_contact_point": float(np.mean(same)) if same else None},
                "training": train_info,
                "moving_bed_10_substeps": moving})
    return res


def storage_variant(B, scene, storage, steps, stream_obj):
    """The same coupled step with 16-bit deviation storage: MLUPS (graph
    replays) and the bulk kernel's roofline fraction (individual launches)."""
    import torch
    sim = build_sim(B, scene, storage, stream_obj.cuda_stream)
    sim.step(1)
    tuning = sim.autotune(os.path.join(tempfile.gettempdir(), "mi_delbm_tune.json"))
    for _ in range(5):
        sim.step(1)
    sim.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream_obj)
    for _ in range(steps):
        sim.step(1)
    ev1.record(stream_obj)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    sim.set_timing(True)
    sim.phase_times(reset=True)
    for _ in range(50):
        sim.step(1)
    bulk_ms, bulk_n = sim.phase_times(reset=True)["bulk"]
    sim.close()
    nx, ny, nz = scene.shape
    ncell = nx * ny * nz
    gbs = BYTES_PER_NODE[storage] * ncell / (bulk_ms / bulk_n * 1e-3) / 1e9
    peak, kind = _peaks()
    return {"value": ncell / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
            "bulk_gbs": gbs, "bulk_frac": gbs / peak, "bytes_per_node": BYTES_PER_NODE[storage], "tuning": tuning,
            "stated_error": STATED_ERROR_C4[storage]}


def dem_ratio(B, scene, storage, steps, stream_obj, nsub=100):
    """The coupled step at the paper's ratio of DEM substeps per LBM step
    (contacts re-detected and particles advanced every substep): MLUPS with
    the fused substep kernel and with one launch sequence per substep."""
    import torch
    out = {"dem_substeps": nsub}
    for name, unfused in (("fused", False), ("per_substep_launches", True)):
        sim = build_sim(B, scene, storage, stream_obj.cuda_stream, dem_substeps=nsub)
        sim.set_schedule(unfused_dem=unfused)
        for _ in range(5):
            sim.step(1)
        sim.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream_obj)
        for _ in range(steps):
            sim.step(1)
        ev1.record(stream_obj)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        sim.close()
        nx, ny, nz = scene.shape
        out[name] = {"value": nx * ny * nz / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms}
    return out


GS_FLOP_PER_PAIR_EPOCH = 27  # field (9) + gradient (18) per (hull point, control point) and epoch
# nominal FP32 rate (SMs x FP32 lanes x FMA x max SM clock), used only when the
# measured peak (mi_measure_fma_peak) is not available
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def gs_bench(B, scenes, n_fits=300, m=2048, epochs=200, seed=11, fp32_peak=FP32_ALU_PEAK_TFLOPS, peak_kind="nominal"):
    """Gradient Search refinement (Algorithm 2) of n_fits models of 8-64
    control points on synthetic bumpy-ellipsoid hulls of m points (the
    300-particle tank's shape range), two descents of `epochs` epochs: fits/s
    and FP32 throughput against the FP32 ALU peak; the FP64 oracle on one fit
    for a few epochs beside it."""
    import ctypes
    import time
    import torch
    from oracle import gs as ogs
    rng = np.random.default_rng(seed)
    hulls, models, planes = [], [], []
    for _ in range(n_fits):
        semi = tuple(rng.uniform(8.0, 16.0, 3))
        H = scenes.ellipsoid_hull(rng, m, semi, bumps=0.15)
        c, k = scenes.gs_start_model(rng, int(rng.integers(8, 65)), semi)
        hulls.append(H)
        models.append(np.concatenate([c, k[:, None]], 1))
        planes.append(scenes.hull_planes(H))
    dev = torch.device("cuda")
    # the generators return float64 arrays of FP32 values: the kernel takes float32
    H = torch.as_tensor(np.concatenate(hulls).astype(np.float32), device=dev)
    M0 = torch.as_tensor(np.concatenate(models).astype(np.float32), device=dev)
    P = torch.as_tensor(np.concatenate(planes).astype(np.float32), device=dev)
    off = lambda arrs: torch.as_tensor(np.concatenate([[0], np.cumsum([len(a) for a in arrs])]).astype(np.int32),
                                       device=dev)
    ho, bo, po = off(hulls), off(models), off(planes)
    nb = [len(a) for a in models]
    active = torch.empty(M0.shape[0], dtype=torch.int32, device=dev)
    loss = torch.empty((n_fits, 2), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    P_ = lambda t: ctypes.c_void_p(t.data_ptr())

    def run(M):
        st = B.lib.mi_gs_fit(n_fits, P_(ho), P_(H), P_(bo), P_(M), P_(po), P_(P), m, max(nb), epochs, 1e-4,
                             P_(active), P_(loss), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, st

    M = M0.clone()
    run(M)
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        M = M0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(M)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    pairs = m * sum(nb)
    flop = 2 * epochs * pairs * GS_FLOP_PER_PAIR_EPOCH
    tflops = flop / (ms * 1e-3) / 1e12
    # oracle: one fit of the same size, a few epochs, scaled to the whole job
    o_ep = 3
    t0 = time.perf_counter()
    c0 = time.process_time()
    ogs.descend(hulls[0].astype(np.float64), models[0][:, :3].astype(np.float64), models[0][:, 3].astype(np.float64),
                o_ep, 1e-4)
    o_wall = time.perf_counter() - t0
    o_cores = cores_used(time.process_time() - c0, o_wall)
    o_s = o_wall * (2 * epochs / o_ep) * (sum(nb) / nb[0])
    ls = loss.cpu().numpy()
    return {"value": n_fits / (ms * 1e-3), "unit": "fits/s", "ms": ms, "fits": n_fits, "hull_points": m,
            "control_points": [int(min(nb)), int(max(nb))], "epochs_per_descent": epochs,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": tflops / fp32_peak, "peak_kind": peak_kind,
                         "flop_per_point_ball_epoch": GS_FLOP_PER_PAIR_EPOCH},
            "loss_after_second_over_first_descent_median": float(np.median(ls[:, 1] / np.maximum(ls[:, 0], 1e-30))),
            "cpu_baseline": {"value": n_fits / o_s, "unit": "fits/s", "cores": o_cores, "kind": "oracle",
                             "sample": "FP64 numpy oracle: %d epochs of one fit, scaled by epochs and control "
                                       "points" % o_ep}}


def ga_bench(B, scenes, n_ind=1200, n_genes=32, m=2048, generations=50, seed=21, fp32_peak=FP32_ALU_PEAK_TFLOPS,
             peak_kind="nominal"):
    """Genetic Algorithm capture (Algorithm 1) with the paper's population of
    1200 individuals: 32-gene models on a 2048-point bumpy-ellipsoid hull,
    `generations` generations: generations/s, fitness evaluations/s and the
    FP32 throughput of the fitness kernel's algorithmic work (9 FLOP per
    (hull point, gene)) against the FP32 ALU peak; the FP64 oracle's fitness
    of one individual beside it."""
    import ctypes
    import time
    import torch
    from oracle import ga as oga
    rng = np.random.default_rng(seed)
    H = scenes.ellipsoid_hull(rng, m, (12.0, 9.0, 7.0), bumps=0.15)
    P = scenes.hull_planes(H)
    bbox = np.concatenate([H.min(0), H.max(0)]).astype(np.float32)
    dev = torch.device("cuda")
    Hd = torch.as_tensor(H.astype(np.float32), device=dev)
    Pd = torch.as_tensor(P.astype(np.float32), device=dev)
    pop = torch.empty((n_ind, n_genes, 4), dtype=torch.float32, device=dev)
    fit = torch.empty(n_ind, dtype=torch.float32, device=dev)
    scratch = torch.empty(int(B.lib.mi_ga_scratch_bytes(n_ind, n_genes)), dtype=torch.uint8, device=dev)
    bb = (ctypes.c_float * 6)(*[float(v) for v in bbox])
    kr = (ctypes.c_float * 2)(2.0, 12.0)
    stream = torch.cuda.current_stream()
    P_ = lambda t: ctypes.c_void_p(t.data_ptr())

    def run(g, init):
        st = B.lib.mi_ga_run(n_ind, n_genes, P_(Hd), m, P_(Pd), int(P.shape[0]), ctypes.cast(bb, ctypes.c_void_p),
                             ctypes.cast(kr, ctypes.c_void_p), 0.05, 0.5, seed, g, init, P_(pop), P_(fit), None, None,
                             P_(scratch), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, st

    run(0, 1)
    torch.cuda.synchronize()
    f0 = float(fit.min().item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run(generations, 0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    evals = n_ind * (generations + 1)
    tflops = evals * m * n_genes * 9 / (ms * 1e-3) / 1e12
    t0 = time.perf_counter()
    c0 = time.process_time()
    oga.fitness(H, pop[0].cpu().numpy())
    o_s = time.perf_counter() - t0
    o_cores = cores_used(time.process_time() - c0, o_s)
    return {"value": generations / (ms * 1e-3), "unit": "generations/s", "ms": ms, "individuals": n_ind,
            "genes": n_genes, "hull_points": m, "generations": generations,
            "fitness_evals_per_s": evals / (ms * 1e-3),
            "roofline": {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": tflops / fp32_peak, "peak_kind": peak_kind, "flop_per_point_gene": 9,
                         "note": "whole generation timed; the fitness kernel's work only"},
            "best_fitness_initial": f0, "best_fitness_final": float(fit[0].item()),
            "cpu_baseline": {"value": 1.0 / o_s, "unit": "fitness evals/s", "cores": o_cores, "kind": "oracle",
                             "sample": "FP64 numpy oracle: one individual's fitness"}}


def shape_bench(B, scenes, n=300, h=0.25, seed=0):
    """Shape descriptors (Sec. 3) of the 300 particle models of the precision
    tank (8-64 control points, radius 8-16 lu) at spacing h: particles/s and
    cell evaluations/s; the oracle on one of them beside it."""
    import time
    import torch
    from oracle import shape as oshape
    sc = scenes.config4(seed=seed, n_particles=n)
    models = [(p.centers, p.k) for p in sc.particles]
    B.shape_descriptors(models[:2], h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = B.shape_descriptors(models, h)
    dt = time.perf_counter() - t0
    cells = sum(int(np.ceil(2.0 * float(np.float32(float(np.sqrt((np.asarray(c, np.float64) ** 2).sum(1)).max()
                                                        + np.sqrt(np.asarray(k, np.float64).sum() / 0.9)))) / h)) ** 3
                for c, k in models)
    # the oracle on the first model at twice the spacing (one eighth of the cells), scaled back
    t1 = time.perf_counter()
    c1 = time.process_time()
    oshape.descriptors(models[0][0], models[0][1], 2 * h)
    o_wall = time.perf_counter() - t1
    o_cores = cores_used(time.process_time() - c1, o_wall)
    o_s = o_wall * 8.0
    return {"value": n / dt, "unit": "particles/s", "s": dt, "particles": n, "h": h,
            "cell_evaluations_per_s": cells / dt, "note": "host wall clock of the binding call (copies included)",
            "sphericity_median": float(np.median([d["sphericity"] for d in out])),
            "csf_median": float(np.median([d["csf"] for d in out])),
            "cpu_baseline": {"value": 1.0 / o_s, "unit": "particles/s", "cores": o_cores, "kind": "oracle",
                             "sample": "numpy oracle: the first particle at twice the spacing, time x 8"}}


C4_KERNELS = ("k_prologue", "k_clear", "k_flag", "k_classify", "k_links_q", "k_refill", "k_bulk", "k_near",
              "k_links_ibb", "k_boundary", "k_dem_prologue", "k_broad_phase", "k_contacts", "k_integrate")
# stated accuracy of each storage on the precision tank: the bounds that
# tests/test_gpu_precision.py asserts on the 128^3 sub-run of that tank
# (eight particles, 30 coupled steps) against the FP64 oracle's reference
STATED_ERROR_C4 = {st: {"velocity_rel_l2_max": bu, "force_rel_max": bf,
                        "asserted_by": "tests/test_gpu_precision.py::test_storage_error_c4_subrun (128^3 sub-run of "
                                       "the 512^3 tank, 8 particles, 30 coupled steps vs the FP64 oracle)"}
                   for st, (bu, bf) in {0: (3.5e-6, 4e-6), 1: (3.5e-4, 2.5e-4), 2: (2.7e-3, 1.5e-3)}.items()}


def c4_leg(B, scenes, stream_obj, steps=100, timed_kernels=20):
    """The precision tank (512^3, 300 particles of 8-64 control points) in
    FP32, FP16-deviation and BF16-deviation storage: coupled-step MLUPS (CUDA
    graph replays, events on the stream), and from a second pass of
    individually launched steps the bulk kernel's HBM fraction inside the step
    and each kernel's event-timed milliseconds per step."""
    import torch
    sc = scenes.config4()
    nx, ny, nz = sc.shape
    ncell = nx * ny * nz
    peak, kind = _peaks()
    out = {"workload": sc.name, "lattice": list(sc.shape), "particles": len(sc.particles),
           "metaballs_min_max": [int(min(len(p.k) for p in sc.particles)), int(max(len(p.k) for p in sc.particles))]}
    for name, st in (("f32", 0), ("f16-dev", 1), ("bf16-dev", 2)):
        t_setup = time.perf_counter()
        sim = build_sim(B, sc, st, stream_obj.cuda_stream)
        sim.step(1)
        tuning = sim.autotune(os.path.join(tempfile.gettempdir(), "mi_delbm_tune.json"))
        for _ in range(5):
            sim.step(1)
        sim.synchronize()
        t_setup = time.perf_counter() - t_setup
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream_obj)
        for _ in range(steps):
            sim.step(1)
        ev1.record(stream_obj)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        sim.set_timing(True)
        sim.phase_times(reset=True)
        for _ in range(timed_kernels):
            sim.step(1)
        kt = {k: sim.kernel_time(k) for k in C4_KERNELS}
        sim.phase_times(reset=True)
        sim.set_timing(False)
        stats = sim.stats()
        sim.close()
        bulk_ms = kt["k_bulk"][0] / max(kt["k_bulk"][1], 1)
        gbs = BYTES_PER_NODE[st] * ncell / (bulk_ms * 1e-3) / 1e9
        out[name] = {"value": ncell / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
                     "bulk_ms": bulk_ms, "bulk_gbs": gbs, "bulk_frac": gbs / peak, "peak_kind": kind,
                     "step_over_bulk": ms / bulk_ms,
                     "kernel_ms_per_step": {k: v[0] / timed_kernels for k, v in kt.items() if v[1]},
                     "boundary_nodes": stats["boundary_nodes"], "links": stats["links"],
                     "candidate_pairs": stats["candidate_pairs"], "tuning": tuning, "setup_s": t_setup,
                     "stated_error": STATED_ERROR_C4[st]}
    return out


def c3_leg(B, scenes, stream_obj, steps=1000):
    """The drafting-kissing-tumbling channel (192x192x768, a 1-ball sphere and
    a 32-ball prolate grain 30 lu apart), FP32: MLUPS with all `steps` steps
    of one call in one CUDA graph launch (a conditional while node over
    two-step bodies) and with one graph launch per step."""
    import torch
    sc = scenes.config3()
    nx, ny, nz = sc.shape
    out = {"workload": sc.name, "lattice": list(sc.shape), "particles": len(sc.particles),
           "metaballs": [int(len(p.k)) for p in sc.particles], "steps": steps}
    for name, loop in (("one_graph_for_all_steps", True), ("one_graph_per_step", False)):
        sim = build_sim(B, sc, 0, stream_obj.cuda_stream)
        sim.set_graphs(True, device_loop=loop)
        sim.step(1)
        sim.autotune(os.path.join(tempfile.gettempdir(), "mi_delbm_tune.json"))
        sim.step(4)
        sim.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = sim.launch_count()
        t0 = time.perf_counter()
        ev0.record(stream_obj)
        if loop:
            sim.step(steps)
        else:
            for _ in range(steps):
                sim.step(1)
        ev1.record(stream_obj)
        host_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        st = [sim.get_particle_state(i) for i in range(len(sc.particles))]
        out[name] = {"value": nx * ny * nz * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms / steps,
                     "kernel_launches": sim.launch_count() - l0, "host_enqueue_s": host_s,
                     "z_after": [float(x["pos"][2]) for x in st]}
        sim.close()
    return out


def measured_alu_peaks(B):
    """FP32 and FP64 FMA throughput of this GPU from the library's own
    microbenchmark (mi_measure_fma_peak)."""
    f32, ms32 = B.measure_fma_peak("fp32")
    f64, ms64 = B.measure_fma_peak("fp64")
    return {"fp32_tflops": f32, "fp64_tflops": f64, "fp32_ms": ms32, "fp64_ms": ms64,
            "how": "mi_measure_fma_peak: 8 independent FMA chains per thread, every SM full, CUDA events"}


def run_mine(args):
    import torch
    from paper_2209_10411_gb300 import replicas
    rank, world, local = replicas.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        replicas.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2209_10411_gb300 import _binding as B
    from paper_2209_10411_gb300 import scenes

    storage = STORAGE[args.storage]
    scene = {"c2": scenes.config2, "c3": scenes.config3, "c4": scenes.config4}[args.config](seed=rank)
    alu = measured_alu_peaks(B) if rank == 0 else None
    if args.lattice:  # smaller profiling case: same particles, positions scaled into the box
        old = np.array(scene.shape, dtype=float)
        scene.shape = tuple(int(v) for v in args.lattice.split(","))
        for p in scene.particles:
            p.pos = scenes.f32(p.pos * np.array(scene.shape) / old)
    stream = torch.cuda.Stream()
    sim = build_sim(B, scene, storage, stream.cuda_stream)
    nx, ny, nz = scene.shape
    ncell = nx * ny * nz
    npart = len(scene.particles)

    # the channel's steps all run in one graph launch (a device-side loop)
    loop = args.config == "c3"
    sim.set_graphs(not args.no_graphs, device_loop=loop)
    sim.step(1)
    tuning = sim.autotune(os.path.join(tempfile.gettempdir(), "mi_delbm_tune.json")) if not args.no_tune else None
    for _ in range(max(3, args.warmup)):
        sim.step(1)
    sim.synchronize()

    # timed region: whole steps (CUDA-graph replays unless --no-graphs)
    clocks = ClockSampler()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    replicas.barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    launches0 = sim.launch_count()
    ev0.record(stream)
    if loop and not args.no_graphs:
        sim.step(args.steps)
    else:
        for _ in range(args.steps):
            sim.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = sim.launch_count() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms = replicas.max_over_ranks(ms, world, device="cuda")
    stats = sim.stats()

    # second timed region, same steps as individual launches bracketed by CUDA
    # events on the stream each kernel runs on: per-kernel durations for the
    # roofline (a graph replays one event pair per node, not one per step)
    k_phase = max(10, min(args.steps, 200))
    sim.set_timing(True)
    sim.phase_times(reset=True)
    for _ in range(k_phase):
        sim.step(1)
    ptimes = sim.phase_times(reset=True)
    sim.set_timing(False)

    # nodes the bulk kernel updates: every node that is neither solid nor boundary
    cls, _ = sim.node_classes()
    n_solid = int(((cls & 1) != 0).sum())
    n_boundary = int(((cls & 2) != 0).sum())
    n_bulk = ncell - n_solid - n_boundary

    value = replicas.aggregate_throughput(ncell * args.steps, world, ms) / 1e6
    bulk_ms, bulk_n = ptimes["bulk"]
    contacts = None
    c2 = args.config == "c2"
    if c2 and not args.no_contacts and rank == 0:
        contacts = contact_solves(B, scenes, args, alu)
    variants = None
    if c2 and storage == 0 and not args.no_variants and rank == 0:
        variants = {name: storage_variant(B, scene, st, max(50, min(args.steps, 200)), stream)
                    for name, st in (("f16-dev", 1), ("bf16-dev", 2))}
        variants["dem_100_substeps"] = dem_ratio(B, scene, storage, 30, stream)
        variants["gs_fit"] = gs_bench(B, scenes, fp32_peak=alu["fp32_tflops"], peak_kind="measured")
        variants["ga_capture"] = ga_bench(B, scenes, fp32_peak=alu["fp32_tflops"], peak_kind="measured")
        variants["shape_descriptors"] = shape_bench(B, scenes)
    c4 = None
    if c2 and not args.no_c4 and rank == 0:
        c4 = c4_leg(B, scenes, stream)
    c3 = None
    if c2 and not args.no_c3 and rank == 0:
        c3 = c3_leg(B, scenes, stream)
    peak, peak_kind = _peaks()
    # the bulk kernel updates every node (boundary nodes are rewritten by the
    # boundary kernel): 19 loads + 19 stores of the stored type per node
    alg_bytes = BYTES_PER_NODE[storage] * ncell
    achieved = alg_bytes / (bulk_ms / bulk_n * 1e-3) / 1e9 if bulk_n else None
    used = tuning if tuning else sim.get_tuning()
    quad = storage != 0 and used.get("bulk_pairs") == 3 and nx % 4 == 0
    traffic = BULK_TRAFFIC.get((storage, quad)) if (nx, ny, nz) == (256, 256, 512) else None
    bulk_name = ("k_bulk_quad16 (D3Q19 stream-collide, four nodes per thread)" if quad
                 else "k_bulk (D3Q19 stream-collide of every node)")

    # end to end through the public API: per step, upload of the particle
    # states from page-locked host memory, the step, and a synchronising read
    # of the hydrodynamic forces and the new states
    states = torch.empty((npart, 13), dtype=torch.float64, pin_memory=True)
    Fh = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
    Th = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
    sim.get_particle_states_ptr(states.data_ptr(), npart)
    sim.synchronize()
    k_e2e = max(10, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        sim.set_particle_states_ptr(states.data_ptr(), npart)
        sim.step(1)
        sim.get_particle_states_ptr(states.data_ptr(), npart)
        sim.forces_ptr(Fh.data_ptr(), Th.data_ptr())
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ncell * k_e2e / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": npart * 13 * 8,
           "d2h_bytes_per_step": npart * (13 + 6) * 8, "steps": k_e2e,
           "api": "set_particle_states + step + get_particle_states + forces per step (host wall clock)"}

    cpu, c2_err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        leg = cpu_leg(B, sim, scene, args.cpu_seconds) if c2 else None
        if leg:
            cpu, c2_err = leg["cpu_baseline"], leg["c2_force_error"]

    config = {"workload": scene.name, "lattice": list(scene.shape), "particles": npart,
              "metaballs": [int(len(p.k)) for p in scene.particles], "storage": args.storage, "tau": scene.tau,
              "boundary_nodes": stats["boundary_nodes"], "links": stats["links"], "solid_nodes": n_solid,
              "l2": "inputs larger than L2 (populations %.2f GB per buffer)" % (19 * ncell * (4 if storage == 0 else 2) / 1e9)}
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE_NAME[storage], "data": "synthetic", "config": config,
           "stated_error": STATED_ERROR_C4[storage],
           "c2_force_error": c2_err,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak if achieved else None, "traffic": traffic,
                        "kernel": bulk_name, "peak_kind": peak_kind,
                        "algorithmic_bytes_per_launch": alg_bytes,
                        "kernel_mlups": ncell / (bulk_ms / bulk_n * 1e-3) / 1e6 if bulk_n else None},
           "phase_ms_per_step": {k: v[0] / k_phase for k, v in ptimes.items() if v[1]},
           "graphs": not args.no_graphs, "tuning": tuning,
           "storage_variants": variants,
           "c4_precision_tank": c4,
           "c3_dkt_channel": c3,
           "contacts": contacts,
           "alu_peaks": alu,
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]}}
    if rank == 0:
        print(json.dumps(out))
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4"])
    ap.add_argument("--storage", default="f32", choices=list(STORAGE))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lattice", default=None, help="nx,ny,nz override (small profiling cases)")
    ap.add_argument("--no-graphs", action="store_true", help="time individual launches instead of graph replays")
    ap.add_argument("--no-contacts", action="store_true", help="skip the contact-solves measurement")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP16/BF16 storage measurements")
    ap.add_argument("--no-c4", action="store_true", help="skip the 512^3 precision-tank measurements")
    ap.add_argument("--no-c3", action="store_true", help="skip the drafting-kissing-tumbling channel measurements")
    ap.add_argument("--schedule", default="default", choices=["default", "overlap"],
                    help="overlap: boundary nodes computed beside the bulk kernel (same bits)")
    ap.add_argument("--small-contact-lattice", action="store_true",
                    help="contact bed on a 16^3 periodic lattice (profiling: same pairs, no walls, little memory)")
    args = ap.parse_args()
    SCHEDULE["overlap"] = args.schedule == "overlap"
    from paper_2209_10411_gb300 import scenes
    sc = {"c2": scenes.config2, "c3": scenes.config3, "c4": scenes.config4}[args.config]()
    # the workload both arms name (the GPU arm adds what its run measures)
    CONFIG.update({"workload": sc.name, "lattice": list(sc.shape), "particles": len(sc.particles),
                   "metaballs": [int(len(p.k)) for p in sc.particles], "storage": args.storage, "tau": sc.tau})
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
