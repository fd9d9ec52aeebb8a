// Engine and C-ABI of libmi_delbm: owns the device state of one lattice and
// its particles, sequences the kernels of one coupled step on one stream.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "engine.h"

using namespace mi;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace mi {
// Message of the last failed handle-less call on this thread (returned by
// mi_delbm_last_error(NULL)).
void set_thread_error(const char* msg) { g_create_error = msg; }
}  // namespace mi

namespace {

// Kernel-launch helper: runs `fn` (which returns a cudaError_t) as one launch
// of `phase`, bracketed by timing events when timing is enabled.
template <class F>
mi_status launch_phase(mi_delbm* h, cudaStream_t st, unsigned phase_bit, const char* kernel, F&& fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = h->event_from_pool();
    b = h->event_from_pool();
    if (!a || !b) return h->fail(MI_ECUDA, "cudaEventCreate failed");
    cudaEventRecord(a, st);
  }
  cudaError_t e = fn();
  h->launches += 1;
  if (e != cudaSuccess) return h->fail(MI_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  if (h->timing) {
    cudaEventRecord(b, st);
    int idx = 0;
    while ((1u << idx) != phase_bit && idx < 7) ++idx;
    h->timed.push_back({idx, a, b, kernel});
  }
  return MI_OK;
}
}  // namespace

// ---------------------------------------------------------------------------
// mi_delbm members
// ---------------------------------------------------------------------------
mi_status mi_delbm::fail(mi_status s, const std::string& msg) {
  err = msg;
  return s;
}

mi_status mi_delbm::cuda_fail(cudaError_t e, const char* what) {
  return fail(MI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* mi_delbm::dalloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (cfg.dev_alloc) {
    p = cfg.dev_alloc(bytes, cfg.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) allocs.push_back({p, bytes});
  return p;
}

void mi_delbm::dfree(void* p) {
  if (!p) return;
  for (size_t i = 0; i < allocs.size(); ++i) {
    if (allocs[i].first == p) {
      if (cfg.dev_free) cfg.dev_free(p, allocs[i].second, cfg.alloc_ctx);
      else cudaFree(p);
      allocs.erase(allocs.begin() + i);
      return;
    }
  }
}

cudaEvent_t mi_delbm::event_from_pool() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

bool mi_delbm::set_device() {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return false;
  if (cur != cfg.device && cudaSetDevice(cfg.device) != cudaSuccess) return false;
  return true;
}

LatticeGeom mi_delbm::geom() const {
  LatticeGeom g;
  g.nx = cfg.nx;
  g.ny = cfg.ny;
  g.nz = cfg.nz;
  for (int a = 0; a < 3; ++a) g.periodic[a] = cfg.periodic[a] ? 1 : 0;
  g.plane = (long long)plane;
  return g;
}

CollideParams mi_delbm::collide_params() const {
  CollideParams p;
  std::memset(&p, 0, sizeof(p));
  p.omega = (float)(1.0 / cfg.tau);
  for (int a = 0; a < 3; ++a) p.force[a] = (float)cfg.fluid_body_force[a];
  for (int f = 0; f < 6; ++f)
    for (int i = 0; i < 19; ++i)
      p.bb_wall[f][i] = (float)(6.0 * wq_d(i) * cfg.rho0 *
                                (cx(i) * cfg.wall_velocity[f][0] + cy(i) * cfg.wall_velocity[f][1] +
                                 cz(i) * cfg.wall_velocity[f][2]));
  p.rho0 = (float)cfg.rho0;
  return p;
}

bool mi_delbm::forcing() const {
  return cfg.fluid_body_force[0] != 0.0 || cfg.fluid_body_force[1] != 0.0 || cfg.fluid_body_force[2] != 0.0;
}

// ---------------------------------------------------------------------------
// Phases
// ---------------------------------------------------------------------------
ParticleLaunch mi_delbm::particle_launch() const {
  ParticleLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.P = dP;
  L.np = n_particles;
  L.balls = dballs;
  L.balls_d = dballs_d;
  L.balls_s = dballs_s;
  L.max_balls_per_particle = max_balls_pp < 2048 ? max_balls_pp : 2048;
  L.cur_buf = owner_cur;
  L.prev_buf = owner_cur ^ 1;
  L.owner_cur = owner[owner_cur];
  L.owner_prev = owner[owner_cur ^ 1];
  L.cls = cls;
  L.stamp = stamp;
  L.ctr = dctr;
  L.facc = facc;
  L.bc_cell = bc_cell;
  L.bc_mask = bc_mask;
  L.bc_loff = bc_loff;
  L.link_bc = link_bc;
  L.link_p = link_p;
  L.link_dir = link_dir;
  L.link_q = link_q;
  L.link_g = link_g;
  L.new_cell = new_cell;
  L.cov_cell = cov_cell;
  L.cover_uncover = cover_uncover ? 1 : 0;
  L.cap_bc = cap_bc;
  L.cap_links = cap_links;
  L.cap_new = cap_new;
  L.flag_off = dblk_off;
  L.cls_off = dblk_off ? dblk_off + cfg.max_particles + 1 : nullptr;
  L.flag_blocks = flag_blocks;
  L.classify_blocks = classify_blocks;
  L.g = geom();
  return L;
}

mi_status mi_delbm::phase_flag(cudaStream_t st) {
  if (n_particles == 0) return MI_OK;
  owner_cur ^= 1;  // the buffer holding the flags of two steps ago becomes current
  ParticleLaunch L = particle_launch();
  mi_status s;
  if ((s = launch_phase(this, st, MI_PHASE_FLAG, "k_prologue", [&] { return launch_prologue(L, st); })) != MI_OK) return s;
  if ((s = launch_phase(this, st, MI_PHASE_FLAG, "k_clear", [&] { return launch_clear(L, st); })) != MI_OK) return s;
  if ((s = launch_phase(this, st, MI_PHASE_FLAG, "k_flag", [&] { return launch_flag(L, st); })) != MI_OK) return s;
  return launch_phase(this, st, MI_PHASE_FLAG, "k_classify", [&] { return launch_classify(L, st); });
}

mi_status mi_delbm::phase_links(cudaStream_t st) {
  if (n_particles == 0) return MI_OK;
  ParticleLaunch L = particle_launch();
  // at most four blocks per SM: the kernel runs beside the bulk kernel,
  // which it slows less with fewer blocks resident at a time
  const int per_sm = tune.list_blocks_per_sm < 4 ? tune.list_blocks_per_sm : 4;
  return launch_phase(this, st, MI_PHASE_LINKS, "k_links_q",
                      [&] { return launch_links_q(L, sm_count * per_sm, st); });
}

static BoundaryLaunch boundary_launch(const mi_delbm* h) {
  BoundaryLaunch L;
  L.pl = h->particle_launch();
  L.A = h->pop[h->cur];
  L.B = h->pop[h->cur ^ 1];
  L.p = h->collide_params();
  L.storage = h->cfg.storage;
  L.forcing = h->forcing();
  L.bb_mode = h->cfg.bb_mode;
  L.grid = h->sm_count * h->tune.list_blocks_per_sm;
  L.tmp = nullptr;
  L.part = h->ibb_part;
  L.part_blocks = h->sm_count * IBB_BLOCKS_PER_SM;
  return L;
}

mi_status mi_delbm::phase_refill(cudaStream_t st) {
  if (n_particles == 0) return MI_OK;
  BoundaryLaunch L = boundary_launch(this);
  return launch_phase(this, st, MI_PHASE_REFILL, "k_refill", [&] { return launch_refill(L, st); });
}

mi_status mi_delbm::phase_near() {
  if (n_particles == 0) return MI_OK;
  BoundaryLaunch L = boundary_launch(this);
  // timed with the boundary phase: the bulk bucket is the lattice-wide kernel alone
  return launch_phase(this, stream, MI_PHASE_BOUNDARY, "k_near", [&] { return launch_near(L, stream); });
}

mi_status mi_delbm::phase_links_ibb(cudaStream_t st) {
  if (n_particles == 0) return MI_OK;
  BoundaryLaunch L = boundary_launch(this);
  return launch_phase(this, st, MI_PHASE_BOUNDARY, "k_links_ibb", [&] { return launch_links_ibb(L, st); });
}

mi_status mi_delbm::phase_boundary() {
  if (n_particles == 0) return MI_OK;
  BoundaryLaunch L = boundary_launch(this);
  return launch_phase(this, stream, MI_PHASE_BOUNDARY, "k_boundary", [&] { return launch_boundary(L, stream); });
}

// Overlapped schedule: the boundary nodes' new values go to bc_tmp on a side
// stream while the bulk kernel writes B (k_boundary reads only A, which the
// refill completes before it, and the links' G, which k_links_ibb writes
// before it on the same stream), and are scattered into B after k_near.
mi_status mi_delbm::phase_boundary_beside(cudaStream_t st) {
  if (n_particles == 0) return MI_OK;
  BoundaryLaunch L = boundary_launch(this);
  L.tmp = bc_tmp;
  return launch_phase(this, st, MI_PHASE_BOUNDARY, "k_boundary", [&] { return launch_boundary(L, st); });
}

mi_status mi_delbm::phase_scatter_boundary() {
  if (n_particles == 0) return MI_OK;
  BoundaryLaunch L = boundary_launch(this);
  L.tmp = bc_tmp;
  return launch_phase(this, stream, MI_PHASE_BOUNDARY, "k_scatter_boundary", [&] { return launch_scatter_boundary(L, stream); });
}

mi_status mi_delbm::phase_integrate(bool with_contacts) {
  if (n_particles == 0) return MI_OK;
  IntegrateLaunch L;
  L.P = dP;
  L.np = n_particles;
  L.facc = facc;
  L.fc = with_contacts ? fc : nullptr;
  for (int a = 0; a < 3; ++a) L.gravity[a] = cfg.gravity[a];
  L.rho0 = cfg.rho0;
  L.dt = 1.0 / cfg.dem_substeps;
  return launch_phase(this, stream, MI_PHASE_INTEGRATE, "k_integrate", [&] { return launch_integrate(L, stream); });
}

mi_status mi_delbm::ensure_contact_buffers() {
  if (contacts_ready) return MI_OK;
  const long long ncap = cfg.max_particles;
  if (ncap > 16384) return fail(MI_ENOTSUP, "contacts: max_particles above 16384 is not supported (pair history size)");
  const long long tri = ncap * (ncap - 1) / 2;
  long long items = std::min<long long>(tri, 64 * ncap) + 6 * ncap;
  cap_items = (unsigned)std::max<long long>(items, 64);
  item_i = (int*)dalloc(sizeof(int) * cap_items);
  item_j = (int*)dalloc(sizeof(int) * cap_items);
  recs = (ContactRec*)dalloc(sizeof(ContactRec) * cap_items);
  hist_pair = (HistEntry*)dalloc(sizeof(HistEntry) * (size_t)std::max<long long>(tri, 1));
  hist_wall = (HistEntry*)dalloc(sizeof(HistEntry) * (size_t)(6 * ncap));
  work = (unsigned*)dalloc(sizeof(unsigned));
  substep = (long long*)dalloc(sizeof(long long));
  bp_pos = (float4*)dalloc(sizeof(float4) * (size_t)std::max<long long>(ncap, 1));
  bp_quat = (float4*)dalloc(sizeof(float4) * (size_t)std::max<long long>(ncap, 1));
  bp_lo = (float4*)dalloc(sizeof(float4) * (size_t)std::max<long long>(ncap, 1));
  bp_vel = (float4*)dalloc(sizeof(float4) * (size_t)std::max<long long>(2 * ncap, 1));
  if (!item_i || !item_j || !recs || !hist_pair || !hist_wall || !work || !substep || !bp_pos || !bp_quat ||
      !bp_lo || !bp_vel)
    return fail(MI_ENOMEM, "contacts: device allocation failed");
  cudaError_t e = cudaMemsetAsync(hist_pair, 0, sizeof(HistEntry) * (size_t)std::max<long long>(tri, 1), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist_wall, 0, sizeof(HistEntry) * (size_t)(6 * ncap), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(substep, 0, sizeof(long long), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return cuda_fail(e, "contacts: initialisation");
  contacts_ready = true;
  return MI_OK;
}

mi_status mi_delbm::ensure_guess_buffers() {
  if (guess_feat) return MI_OK;
  mi_status s = ensure_contact_buffers();
  if (s != MI_OK) return s;
  guess_feat = (float*)dalloc(sizeof(float) * 64 * (size_t)cap_items);
  guess_pred = (float*)dalloc(sizeof(float) * 4 * (size_t)cap_items);
  mlp_image = dalloc(mlp_image_total());
  if (!guess_feat || !guess_pred || !mlp_image) return fail(MI_ENOMEM, "learned guess: device allocation failed");
  return MI_OK;
}

static ContactLaunch contact_launch(const mi_delbm* h) {
  ContactLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.P = h->dP;
  L.np = h->n_particles;
  L.ncap = h->cfg.max_particles;
  L.balls = h->dballs;
  L.ctr = h->dctr;
  L.work = h->work;
  L.item_i = h->item_i;
  L.item_j = h->item_j;
  L.cap_items = h->cap_items;
  L.recs = h->recs;
  L.hist_pair = h->hist_pair;
  L.hist_wall = h->hist_wall;
  L.fcacc = h->fc;
  L.substep = h->substep;
  L.cp.kn = h->cfg.kn;
  L.cp.kt = h->cfg.kt;
  L.cp.eta_n = h->cfg.eta_n;
  L.cp.eta_t = h->cfg.eta_t;
  L.cp.mu_s = h->cfg.mu_s;
  L.cp.dt = 1.0 / h->cfg.dem_substeps;
  L.cp.margin = 1.0;
  L.pf = h->bp_pos;
  L.qf = h->bp_quat;
  L.plo = h->bp_lo;
  L.vw = h->bp_vel;
  L.cf = {(float)L.cp.kn, (float)L.cp.kt, (float)L.cp.eta_n, (float)L.cp.eta_t, (float)L.cp.mu_s, (float)L.cp.dt};
  L.learned = h->learned ? 1 : 0;
  L.warm = h->warm ? 1 : 0;
  L.feat = h->guess_feat;
  L.pred = h->guess_pred;
  for (int a = 0; a < 3; ++a) L.cp.periodic[a] = h->cfg.periodic[a] ? 1 : 0;
  L.cp.n[0] = h->cfg.nx;
  L.cp.n[1] = h->cfg.ny;
  L.cp.n[2] = h->cfg.nz;
  // 128-thread blocks of <= 85 registers: six fit on an SM; never more warps
  // than there can be candidates (pairs and walls), so that a few particles
  // do not take every SM's registers from the kernels running beside
  const long long npl = h->n_particles;
  const long long most = std::min<long long>(npl * (npl - 1) / 2 + 6 * npl, (long long)h->cap_items);
  L.grid = (int)std::max<long long>(1, std::min<long long>((long long)h->sm_count * 6, (most + 3) / 4));
  return L;
}

mi_status mi_delbm::phase_contact(cudaStream_t st) {
  if (n_particles == 0) return MI_OK;
  mi_status s = ensure_contact_buffers();
  if (s != MI_OK) return s;
  if (learned && (s = ensure_guess_buffers()) != MI_OK) return s;
  ContactLaunch L = contact_launch(this);
  if ((s = launch_phase(this, st, MI_PHASE_CONTACT, "k_dem_prologue", [&] { return launch_dem_prologue(L, st); })) != MI_OK) return s;
  if ((s = launch_phase(this, st, MI_PHASE_CONTACT, "k_broad_phase", [&] { return launch_broad_phase(L, st); })) != MI_OK) return s;
  if (learned) {
    // features of the candidates, then the MLP on as many rows as the broad phase found
    if ((s = launch_phase(this, st, MI_PHASE_CONTACT, "k_item_features", [&] { return launch_item_features(L, st); })) != MI_OK) return s;
    if ((s = launch_phase(this, st, MI_PHASE_CONTACT, "k_mlp_tc", [&] {
           return mlp_tc_infer(static_cast<unsigned char*>(mlp_image) + mlp_image_bytes(), guess_feat,
                               (int)cap_items, &dctr->n_pairs, guess_pred, &dctr->status, STATUS_GUESS_TIMEOUT, st,
                               guess_wait_limit, guess_stall);
         })) != MI_OK)
      return s;
  }
  return launch_phase(this, st, MI_PHASE_CONTACT, "k_contacts", [&] { return launch_contacts(L, st); });
}

mi_status mi_delbm::phase_bulk() {
  BulkLaunch L;
  L.A = pop[cur];
  L.B = pop[cur ^ 1];
  L.g = geom();
  L.p = collide_params();
  L.storage = cfg.storage;
  L.forcing = forcing();
  L.block_x = tune.bulk_block_x;
  L.rows = tune.bulk_rows;
  L.pairs = tune.bulk_pairs != 0;
  L.pair_mode = tune.bulk_pairs;
  return launch_phase(this, stream, MI_PHASE_BULK, "k_bulk", [&] { return launch_bulk(L, stream); });
}

mi_status mi_delbm::phase_swap() {
  cur ^= 1;
  step_index += 1;
  return MI_OK;
}

// The phases of one step.  The bulk stream-collide of every node runs on the
// handle's stream; concurrently, on high-priority side streams, run the
// particle chain (flag, classify, refill; the wall fractions fork off it and
// the links' bounce-back and momentum exchange follow both) and the first
// DEM substep's contacts (they read only the particle state, which changes at
// the rigid-body update).  After the bulk kernel and the particle chain meet,
// the neighbours of uncovered nodes are recomputed (k_near), then the
// boundary nodes, then the DEM substeps.
mi_status mi_delbm::run_phases(unsigned phases) {
  mi_status s = MI_OK;
  const bool particles = n_particles > 0;
  const bool contact_branch = particles && (phases & MI_PHASE_CONTACT);
  const bool chain = particles && (phases & (MI_PHASE_FLAG | MI_PHASE_LINKS | MI_PHASE_REFILL));
  const bool links_branch = particles && (phases & MI_PHASE_LINKS);
  // overlapped boundary schedule: needs the whole chain, the wall fractions and the bulk kernel in this call
  const bool beside = overlap_boundary && links_branch && (phases & MI_PHASE_BOUNDARY) && (phases & MI_PHASE_BULK) &&
                      (phases & MI_PHASE_FLAG) && (phases & MI_PHASE_REFILL);
  // the links' bounce-back on the chain: needs the wall fractions and the refill in this call
  const bool ibb_beside = (links_beside || beside) && chain && links_branch && (phases & MI_PHASE_BOUNDARY) &&
                          (phases & MI_PHASE_REFILL);
  if (contact_branch) {
    if ((s = ensure_contact_buffers()) != MI_OK) return s;
    if ((s = fork(stream, aux[1], 0)) != MI_OK) return s;
    if ((s = phase_contact(aux[1])) != MI_OK) return s;
    if ((s = join_record(aux[1], 0)) != MI_OK) return s;
  }
  if (chain) {
    if ((s = fork(stream, aux[2], 2)) != MI_OK) return s;
    if ((phases & MI_PHASE_FLAG) && (s = phase_flag(aux[2])) != MI_OK) return s;
    if (links_branch) {
      if ((s = fork(aux[2], aux[0], 1)) != MI_OK) return s;
      if ((s = phase_links(aux[0])) != MI_OK) return s;
      if ((s = join_record(aux[0], 1)) != MI_OK) return s;
    }
    if ((phases & MI_PHASE_REFILL) && (s = phase_refill(aux[2])) != MI_OK) return s;
    if (ibb_beside) {
      // after the refill and the wall fractions: the links' bounce-back, and in
      // the overlapped schedule the boundary nodes too
      cudaError_t e = cudaEventRecord(ev_join[1], aux[0]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(aux[2], ev_join[1], 0);
      if (e != cudaSuccess) return cuda_fail(e, "join");
      if ((s = phase_links_ibb(aux[2])) != MI_OK) return s;
      if (beside && (s = phase_boundary_beside(aux[2])) != MI_OK) return s;
    }
    if ((s = join_record(aux[2], 2)) != MI_OK) return s;
  }
  if ((phases & MI_PHASE_BULK) && (s = phase_bulk()) != MI_OK) return s;
  if (chain && (s = join_wait(2)) != MI_OK) return s;
  if ((phases & MI_PHASE_BULK) && (s = phase_near()) != MI_OK) return s;
  if (beside) {
    if ((s = phase_scatter_boundary()) != MI_OK) return s;
  } else {
    if (links_branch && (s = join_wait(1)) != MI_OK) return s;
    if ((phases & MI_PHASE_BOUNDARY) && !ibb_beside && (s = phase_links_ibb(stream)) != MI_OK) return s;
    if ((phases & MI_PHASE_BOUNDARY) && (s = phase_boundary()) != MI_OK) return s;
  }
  if ((phases & MI_PHASE_SWAP) && (s = phase_swap()) != MI_OK) return s;
  if (contact_branch && (s = join_wait(0)) != MI_OK) return s;
  if (phases & (MI_PHASE_CONTACT | MI_PHASE_INTEGRATE)) {
    // several substeps of a few particles: one fused kernel (plain or warm start)
    const bool fused = (phases & MI_PHASE_CONTACT) && (phases & MI_PHASE_INTEGRATE) && cfg.dem_substeps > 1 &&
                       n_particles > 0 && n_particles <= FUSED_DEM_MAX_PARTICLES && !learned && !unfused_dem;
    if (fused) return phase_dem_fused();
    for (int k = 0; k < cfg.dem_substeps; ++k) {
      if (k > 0 && (phases & MI_PHASE_CONTACT) && (s = phase_contact(stream)) != MI_OK) return s;
      if ((phases & MI_PHASE_INTEGRATE) && (s = phase_integrate((phases & MI_PHASE_CONTACT) != 0)) != MI_OK) return s;
    }
  }
  return MI_OK;
}

mi_status mi_delbm::phase_dem_fused() {
  mi_status s = ensure_contact_buffers();
  if (s != MI_OK) return s;
  ContactLaunch L = contact_launch(this);
  IntegrateLaunch I;
  I.P = dP;
  I.np = n_particles;
  I.facc = facc;
  I.fc = fc;
  for (int a = 0; a < 3; ++a) I.gravity[a] = cfg.gravity[a];
  I.rho0 = cfg.rho0;
  I.dt = 1.0 / cfg.dem_substeps;
  return launch_phase(this, stream, MI_PHASE_INTEGRATE, "k_dem_substeps",
                      [&] { return launch_dem_substeps(L, I, cfg.dem_substeps, stream); });
}

void mi_delbm::invalidate_graphs() {
  for (int k = 0; k < 4; ++k) {
    if (gexec[k]) cudaGraphExecDestroy(gexec[k]);
    gexec[k] = nullptr;
    glaunches[k] = 0;
    if (gloop[k]) cudaGraphExecDestroy(gloop[k]);
    gloop[k] = nullptr;
    gloop_launches[k] = 0;
  }
}

namespace {
__global__ void k_loop_set(int* count, long long pairs) { *count = (int)pairs; }
// The last node of the loop body: one step pair done; run the body again
// while pairs are left.
__global__ void k_loop_tail(int* count, cudaGraphConditionalHandle h) {
  const int left = *count - 1;
  *count = left;
  cudaGraphSetConditional(h, left > 0 ? 1u : 0u);
}
}  // namespace

// `pairs` step pairs as one graph launch: a conditional while node whose body
// (captured from the same run_phases() as the eager path, twice, so that
// both buffer parities are in it) ends with a kernel that counts the pairs
// down on the device.  The host state advances by 2 pairs steps; the
// buffer parities return to where they were.
mi_status mi_delbm::loop_steps(long long pairs) {
  if (pairs <= 0) return MI_OK;
  if (pairs > 0x7FFFFFFF) return fail(MI_EINVAL, "mi_delbm_step: too many steps for one device loop");
  const int key = (cur & 1) | ((owner_cur & 1) << 1);
  if (!loop_count) {
    loop_count = (int*)dalloc(sizeof(int));
    if (!loop_count) return fail(MI_ENOMEM, "device loop: counter allocation failed");
  }
  if (!gloop[key]) {
    if (n_particles > 0) {
      mi_status s = ensure_contact_buffers();
      if (s != MI_OK) return s;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    cudaGraphConditionalHandle hnd;
    e = cudaGraphConditionalHandleCreate(&hnd, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "device loop: conditional node");
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    const int c0 = cur, o0 = owner_cur;
    const long long s0 = step_index, l0 = launches;
    e = cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "cudaStreamBeginCaptureToGraph");
    }
    mi_status st = run_phases(MI_PHASE_ALL);
    if (st == MI_OK) st = run_phases(MI_PHASE_ALL);
    if (st == MI_OK) {
      k_loop_tail<<<1, 1, 0, stream>>>(loop_count, hnd);
      launches += 1;
      if (cudaGetLastError() != cudaSuccess) st = fail(MI_ECUDA, "device loop: tail launch failed");
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(stream, &captured);
    gloop_launches[key] = launches - l0;
    cur = c0;
    owner_cur = o0;
    step_index = s0;
    launches = l0;
    if (st != MI_OK || e2 != cudaSuccess) {
      cudaGraphDestroy(g);
      return st != MI_OK ? st : cuda_fail(e2, "cudaStreamEndCapture (device loop)");
    }
    e = cudaGraphInstantiate(&gloop[key], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gloop[key] = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate (device loop)");
    }
  }
  k_loop_set<<<1, 1, 0, stream>>>(loop_count, pairs);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaGraphLaunch(gloop[key], stream);
  if (e != cudaSuccess) return cuda_fail(e, "device loop launch");
  launches += 1 + pairs * gloop_launches[key];
  step_index += 2 * pairs;
  return MI_OK;
}

// One full step replayed from a CUDA graph.  A step alternates the population
// buffers and (with particles) the owner buffers, so at most four graphs exist,
// keyed by those two parities; each is captured on first use from the same
// run_phases() the eager path runs.  Nothing allocates inside a capture: the
// buffers a step needs are created first.
mi_status mi_delbm::graph_step() {
  const int key = (cur & 1) | ((owner_cur & 1) << 1);
  if (!gexec[key]) {
    if (n_particles > 0) {
      mi_status s = ensure_contact_buffers();
      if (s != MI_OK) return s;
    }
    const int c0 = cur, o0 = owner_cur;
    const long long s0 = step_index, l0 = launches;
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    mi_status st = run_phases(MI_PHASE_ALL);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(stream, &g);
    glaunches[key] = launches - l0;
    cur = c0;
    owner_cur = o0;
    step_index = s0;
    launches = l0;
    if (st != MI_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&gexec[key], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gexec[key] = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  cudaError_t e = cudaGraphLaunch(gexec[key], stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  launches += glaunches[key];
  cur ^= 1;
  step_index += 1;
  if (n_particles > 0) owner_cur ^= 1;
  return MI_OK;
}

mi_status mi_delbm::fork(cudaStream_t from, cudaStream_t to, int slot) {
  cudaError_t e = cudaEventRecord(ev_fork[slot], from);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev_fork[slot], 0);
  if (e != cudaSuccess) return cuda_fail(e, "fork");
  return MI_OK;
}

mi_status mi_delbm::join_record(cudaStream_t from, int slot) {
  cudaError_t e = cudaEventRecord(ev_join[slot], from);
  if (e != cudaSuccess) return cuda_fail(e, "join");
  return MI_OK;
}

mi_status mi_delbm::join_wait(int slot) {
  cudaError_t e = cudaStreamWaitEvent(stream, ev_join[slot], 0);
  if (e != cudaSuccess) return cuda_fail(e, "join");
  return MI_OK;
}

mi_status mi_delbm::sync(const char* what) {
  if (!set_device()) return fail(MI_ECUDA, "cudaSetDevice failed");
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  return MI_OK;
}

mi_status mi_delbm::check_status(bool clear) {
  if (!particles_ready) return MI_OK;
  DevCounters c;
  cudaError_t e = cudaMemcpyAsync(&c, dctr, sizeof(c), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading device status");
  if (c.status & STATUS_GUESS_TIMEOUT) {
    if (clear) {
      unsigned zero = 0;
      cudaMemcpyAsync(&dctr->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, stream);
      cudaStreamSynchronize(stream);
    }
    return fail(MI_ETIMEOUT, "the learned-guess MLP kernel gave up a bounded wait (its rows were marked NaN and the "
                             "contacts fell back to plain Newton)");
  }
  const unsigned bad = c.status & (STATUS_BC_OVERFLOW | STATUS_LINK_OVERFLOW | STATUS_NEW_OVERFLOW |
                                   STATUS_PAIR_OVERFLOW | STATUS_CONTACT_OVERFLOW);
  if (clear && c.status) {
    unsigned zero = 0;
    cudaMemcpyAsync(&dctr->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, stream);
    cudaStreamSynchronize(stream);
  }
  if (bad & (STATUS_BC_OVERFLOW | STATUS_LINK_OVERFLOW | STATUS_NEW_OVERFLOW)) {
    // the counters hold the full counts (appends are counted before the
    // capacity test): the lists grow to them before the next step
    need_bc = std::max(need_bc, c.n_bc);
    need_links = std::max(need_links, c.n_links);
    need_new = std::max(need_new, std::max(c.n_new, c.n_cov));
  }
  if (bad) {
    return fail(MI_ECAPACITY, "a device list overflowed during the step (status bits " + std::to_string(bad) +
                                  "; boundary nodes " + std::to_string(c.n_bc) + "/" + std::to_string(cap_bc) +
                                  ", links " + std::to_string(c.n_links) + "/" + std::to_string(cap_links) +
                                  ", uncovered " + std::to_string(c.n_new) + "/" + std::to_string(cap_new) +
                                  ", covered " + std::to_string(c.n_cov) + "/" + std::to_string(cap_new) + ")");
  }
  return MI_OK;
}

// Before a step: lists that a previous step overflowed grow to what it
// needed plus a quarter (the graphs, which hold the old list pointers, are
// captured again).
mi_status mi_delbm::grow_lists_if_needed() {
  if (need_bc <= cap_bc && need_links <= cap_links && need_new <= cap_new) return MI_OK;
  auto grown = [](unsigned need, unsigned cap) -> unsigned {
    if (need <= cap) return cap;
    const unsigned long long g = (unsigned long long)need + need / 4 + 64;
    return (unsigned)std::min<unsigned long long>(g, 0xFFFFFFF0ull);
  };
  mi_status s = ensure_list_capacity(grown(need_bc, cap_bc), grown(need_links, cap_links), grown(need_new, cap_new));
  if (s != MI_OK) return s;
  invalidate_graphs();
  return MI_OK;
}

mi_status mi_delbm::ensure_particle_buffers() {
  if (particles_ready) return MI_OK;
  const int np = cfg.max_particles > 0 ? cfg.max_particles : 1;
  const int nb = cfg.max_balls > 0 ? cfg.max_balls : 1;
  owner[0] = (uint32_t*)dalloc(ncell * 4);
  owner[1] = (uint32_t*)dalloc(ncell * 4);
  stamp = (uint32_t*)dalloc(ncell * 4);
  dctr = (DevCounters*)dalloc(sizeof(DevCounters));
  facc = (long long*)dalloc(sizeof(long long) * 6 * np);
  fc = (long long*)dalloc(sizeof(long long) * 6 * np);
  dP = (DevParticle*)dalloc(sizeof(DevParticle) * np);
  dballs = (float4*)dalloc(sizeof(float4) * nb);
  dballs_d = (double*)dalloc(sizeof(double) * 4 * nb);
  dballs_s = (float4*)dalloc(sizeof(float4) * 2 * nb);
  dblk_off = (int*)dalloc(sizeof(int) * 2 * ((size_t)np + 1));
  if (!dblk_off) return fail(MI_ENOMEM, "particle buffers: device allocation failed");
  if (np <= IBB_SHARED_PARTICLES) {
    ibb_part = (long long*)dalloc(sizeof(long long) * 6 * (size_t)np * sm_count * IBB_BLOCKS_PER_SM);
    if (!ibb_part) return fail(MI_ENOMEM, "particle buffers: device allocation failed");
  }
  if (!owner[0] || !owner[1] || !stamp || !dctr || !facc || !fc || !dP || !dballs || !dballs_d || !dballs_s)
    return fail(MI_ENOMEM, "particle buffers: device allocation failed");
  cudaError_t e = cudaMemsetAsync(owner[0], 0xFF, ncell * 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(owner[1], 0xFF, ncell * 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(stamp, 0, ncell * 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dctr, 0, sizeof(DevCounters), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(facc, 0, sizeof(long long) * 6 * np, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(fc, 0, sizeof(long long) * 6 * np, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "particle buffers: initialisation");
  particles_ready = true;
  return MI_OK;
}

mi_status mi_delbm::ensure_list_capacity(unsigned bc, unsigned links, unsigned nnew) {
  if (bc <= cap_bc && links <= cap_links && nnew <= cap_new) return MI_OK;
  mi_status s = sync("list reallocation");
  if (s != MI_OK) return s;
  bc = bc > cap_bc ? bc : cap_bc;
  links = links > cap_links ? links : cap_links;
  nnew = nnew > cap_new ? nnew : cap_new;
  dfree(bc_cell); dfree(bc_mask); dfree(bc_loff); dfree(link_bc); dfree(link_p); dfree(link_dir);
  dfree(link_q); dfree(link_g); dfree(new_cell); dfree(cov_cell); dfree(bc_tmp);
  bc_cell = (uint32_t*)dalloc(4ull * bc);
  bc_mask = (uint32_t*)dalloc(4ull * bc);
  bc_loff = (uint32_t*)dalloc(4ull * bc);
  link_bc = (uint32_t*)dalloc(4ull * links);
  link_p = (uint32_t*)dalloc(4ull * links);
  link_dir = (uint8_t*)dalloc(1ull * links);
  link_q = (float*)dalloc(4ull * links);
  link_g = (float*)dalloc(4ull * links);
  new_cell = (uint32_t*)dalloc(4ull * nnew);
  cov_cell = (uint32_t*)dalloc(4ull * nnew);
  bc_tmp = dalloc(19ull * store_bytes(cfg.storage) * bc);
  if (!bc_cell || !bc_mask || !bc_loff || !link_bc || !link_p || !link_dir || !link_q || !link_g || !new_cell ||
      !cov_cell ||
      !bc_tmp) {
    cap_bc = cap_links = cap_new = 0;
    return fail(MI_ENOMEM, "link lists: device allocation failed");
  }
  cap_bc = bc;
  cap_links = links;
  cap_new = nnew;
  return MI_OK;
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

int mi_delbm_abi_version(void) { return MI_DELBM_ABI_VERSION; }
size_t mi_delbm_config_size(void) { return sizeof(mi_delbm_config); }

void mi_delbm_config_init(mi_delbm_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = c->ny = c->nz = 64;
  c->tau = 0.8;
  c->rho0 = 1.0;
  c->storage = MI_STORE_F32;
  c->bb_mode = MI_BB_IBB;
  c->dem_substeps = 1;
  c->kn = 1.0;
  c->kt = 2.0 / 7.0;
  c->eta_n = 0.0;
  c->eta_t = 0.0;
  c->mu_s = 0.4;
  c->guess_mode = MI_GUESS_PLAIN;
  c->check_overlap = 0;
  c->max_particles = 1024;
  c->max_balls = 65536;
  c->cuda_stream = nullptr;
  c->device = 0;
}

mi_status mi_delbm_create(const mi_delbm_config* cfg, mi_delbm** out) {
  if (!cfg || !out) {
    g_create_error = "mi_delbm_create: null argument";
    return MI_EINVAL;
  }
  *out = nullptr;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->nx > 65535 * 256 || cfg->ny > 65535 ||
      cfg->nz > 65535) {
    g_create_error = "mi_delbm_create: lattice sizes must be >= 1 (ny, nz <= 65535)";
    return MI_EINVAL;
  }
  const long long ncell = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (ncell > (1LL << 31) - 1) {
    g_create_error = "mi_delbm_create: more than 2^31-1 nodes";
    return MI_EINVAL;
  }
  if (!(cfg->tau > 0.5)) {
    g_create_error = "mi_delbm_create: tau must be > 1/2";
    return MI_EINVAL;
  }
  if (!(cfg->rho0 > 0.0)) {
    g_create_error = "mi_delbm_create: rho0 must be > 0";
    return MI_EINVAL;
  }
  if (cfg->storage < MI_STORE_F32 || cfg->storage > MI_STORE_BF16_DEV) {
    g_create_error = "mi_delbm_create: unknown storage";
    return MI_EINVAL;
  }
  if (cfg->bb_mode != MI_BB_IBB && cfg->bb_mode != MI_BB_LADD) {
    g_create_error = "mi_delbm_create: unknown bb_mode";
    return MI_EINVAL;
  }
  if (cfg->dem_substeps < 1 || cfg->max_particles < 0 || cfg->max_balls < 0 || cfg->max_particles > 65535) {
    g_create_error = "mi_delbm_create: dem_substeps must be >= 1, capacities >= 0, max_particles <= 65535";
    return MI_EINVAL;
  }
  if (cfg->guess_mode != MI_GUESS_PLAIN && cfg->guess_mode != MI_GUESS_WARM) {
    g_create_error = "mi_delbm_create: guess_mode must be MI_GUESS_PLAIN or MI_GUESS_WARM (load a learned guess "
                     "with mi_delbm_set_guess)";
    return MI_EINVAL;
  }
  if ((cfg->dev_alloc == nullptr) != (cfg->dev_free == nullptr)) {
    g_create_error = "mi_delbm_create: dev_alloc and dev_free must be given together";
    return MI_EINVAL;
  }
  mi_delbm* h = new (std::nothrow) mi_delbm();
  if (!h) {
    g_create_error = "mi_delbm_create: out of host memory";
    return MI_ENOMEM;
  }
  h->cfg = *cfg;
  h->warm = cfg->guess_mode == MI_GUESS_WARM;
  if (!h->set_device()) {
    g_create_error = "mi_delbm_create: cudaSetDevice failed";
    delete h;
    return MI_ECUDA;
  }
  if (cfg->cuda_stream) {
    h->stream = (cudaStream_t)cfg->cuda_stream;
    h->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      g_create_error = "mi_delbm_create: cudaStreamCreate failed";
      delete h;
      return MI_ECUDA;
    }
    h->own_stream = true;
  }
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  for (int i = 0; i < 3; ++i) {
    if (cudaStreamCreateWithPriority(&h->aux[i], cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
      g_create_error = "mi_delbm_create: side stream / event creation failed";
      mi_delbm_destroy(h);
      return MI_ECUDA;
    }
  }
  h->ncell = (size_t)ncell;
  h->plane = (h->ncell + 63) / 64 * 64;  // 256-byte aligned planes for every storage
  h->esize = store_bytes(cfg->storage);
  const size_t pop_bytes = 19 * h->plane * h->esize;
  h->pop[0] = h->dalloc(pop_bytes);
  h->pop[1] = h->dalloc(pop_bytes);
  h->cls = (uint8_t*)h->dalloc(h->ncell);
  if (!h->pop[0] || !h->pop[1] || !h->cls) {
    g_create_error = "mi_delbm_create: device allocation failed (" + std::to_string(2 * pop_bytes + h->ncell) + " bytes)";
    mi_delbm_destroy(h);
    return MI_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(h->cls, 0, h->ncell, h->stream);
  if (e == cudaSuccess) e = launch_fill_rest(h->pop[0], h->geom(), cfg->storage, (float)cfg->rho0, h->stream);
  if (e == cudaSuccess) e = launch_fill_rest(h->pop[1], h->geom(), cfg->storage, (float)cfg->rho0, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    g_create_error = std::string("mi_delbm_create: initialisation failed: ") + cudaGetErrorString(e);
    mi_delbm_destroy(h);
    return MI_ECUDA;
  }
  h->tune.bulk_block_x = cfg->nx >= 256 ? 128 : (cfg->nx >= 128 ? 64 : 32);
  h->tune.bulk_rows = 1;
  h->tune.bulk_pairs = 0;
  if (cfg->storage != MI_STORE_F32 && cfg->nx % 4 == 0) {
    // 16-bit storages: four nodes per thread with 64-bit accesses
    h->tune.bulk_pairs = 3;
    h->tune.bulk_block_x = cfg->nx >= 256 ? 64 : 32;
  }
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device) == cudaSuccess && sms > 0)
      h->sm_count = sms;
  }
  *out = h;
  return MI_OK;
}

void mi_delbm_destroy(mi_delbm* h) {
  if (!h) return;
  h->set_device();
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& t : h->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  h->invalidate_graphs();
  for (int i = 0; i < 3; ++i) {
    if (h->aux[i]) cudaStreamSynchronize(h->aux[i]);
    if (h->aux[i]) cudaStreamDestroy(h->aux[i]);
    if (h->ev_fork[i]) cudaEventDestroy(h->ev_fork[i]);
    if (h->ev_join[i]) cudaEventDestroy(h->ev_join[i]);
  }
  while (!h->allocs.empty()) h->dfree(h->allocs.back().first);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* mi_delbm_last_error(const mi_delbm* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

mi_status mi_delbm_step(mi_delbm* h, int n_steps) {
  if (!h) return MI_EINVAL;
  if (n_steps < 0) return h->fail(MI_EINVAL, "mi_delbm_step: n_steps < 0");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  mi_status s = h->grow_lists_if_needed();
  if (s != MI_OK) return s;
  int n = 0;
  if (h->use_graphs && h->loop_graphs && !h->timing && n_steps >= 2) {
    if ((s = h->loop_steps(n_steps / 2)) != MI_OK) return s;
    n = 2 * (n_steps / 2);
  }
  for (; n < n_steps; ++n) {
    s = (h->use_graphs && !h->timing) ? h->graph_step() : h->run_phases(MI_PHASE_ALL);
    if (s != MI_OK) return s;
  }
  return MI_OK;
}

mi_status mi_delbm_synchronize(mi_delbm* h) {
  if (!h) return MI_EINVAL;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_synchronize");
  return MI_OK;
}

mi_status mi_delbm_step_phases(mi_delbm* h, unsigned phases) {
  if (!h) return MI_EINVAL;
  if (phases & ~0xFFu) return h->fail(MI_EINVAL, "mi_delbm_step_phases: unknown phase bits");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  mi_status s = h->grow_lists_if_needed();
  if (s != MI_OK) return s;
  return h->run_phases(phases);
}

mi_status mi_delbm_reserve_lists(mi_delbm* h, size_t boundary_nodes, size_t links, size_t new_nodes) {
  if (!h) return MI_EINVAL;
  if (boundary_nodes < 1 || links < 1 || new_nodes < 1 || boundary_nodes > 0xFFFFFFF0ull || links > 0xFFFFFFF0ull ||
      new_nodes > 0xFFFFFFF0ull)
    return h->fail(MI_EINVAL, "mi_delbm_reserve_lists: each capacity must be in 1 .. 2^32 - 16");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  if (!h->particles_ready) {
    mi_status s = h->ensure_particle_buffers();
    if (s != MI_OK) return s;
  }
  // exactly these sizes: drop the current lists first so that they may shrink
  mi_status s = h->sync("mi_delbm_reserve_lists");
  if (s != MI_OK) return s;
  h->dfree(h->bc_cell); h->dfree(h->bc_mask); h->dfree(h->bc_loff); h->dfree(h->link_bc); h->dfree(h->link_p);
  h->dfree(h->link_dir); h->dfree(h->link_q); h->dfree(h->link_g); h->dfree(h->new_cell); h->dfree(h->cov_cell);
  h->dfree(h->bc_tmp);
  h->bc_cell = h->bc_mask = h->bc_loff = h->link_bc = h->link_p = h->new_cell = h->cov_cell = nullptr;
  h->link_dir = nullptr;
  h->link_q = nullptr;
  h->link_g = nullptr;
  h->bc_tmp = nullptr;
  h->cap_bc = h->cap_links = h->cap_new = 0;
  h->need_bc = h->need_links = h->need_new = 0;
  s = h->ensure_list_capacity((unsigned)boundary_nodes, (unsigned)links, (unsigned)new_nodes);
  h->invalidate_graphs();
  return s;
}

mi_status mi_delbm_set_guess_wait(mi_delbm* h, unsigned wait_rounds, int stall) {
  if (!h) return MI_EINVAL;
  h->guess_wait_limit = wait_rounds;
  h->guess_stall = stall ? 1 : 0;
  h->invalidate_graphs();
  return MI_OK;
}

mi_status mi_delbm_check(mi_delbm* h, mi_delbm_health* out) {
  if (!h || !out) return MI_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->first_bad_node = -1;
  out->first_bad_particle = -1;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  if (!h->check_buf) {
    h->check_buf = (long long*)h->dalloc(2 * sizeof(long long));
    if (!h->check_buf) return h->fail(MI_ENOMEM, "mi_delbm_check: device allocation failed");
  }
  const uint32_t* own = h->particles_ready && h->n_particles > 0 ? h->owner[h->owner_cur] : nullptr;
  cudaError_t e = launch_check(h->pop[h->cur], h->geom(), h->cfg.storage, own, h->check_buf, h->sm_count, h->stream);
  long long res[2] = {0, -1};
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, h->check_buf, sizeof(res), cudaMemcpyDeviceToHost, h->stream);
  std::vector<DevParticle> parts((size_t)h->n_particles);
  if (e == cudaSuccess && h->n_particles > 0)
    e = cudaMemcpyAsync(parts.data(), h->dP, sizeof(DevParticle) * parts.size(), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_check");
  out->bad_populations = res[0];
  out->first_bad_node = res[0] > 0 ? res[1] : -1;
  for (int p = 0; p < h->n_particles; ++p) {
    const DevParticle& P = parts[p];
    bool ok = true;
    for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(P.pos[a]) && std::isfinite(P.vel[a]) && std::isfinite(P.omega[a]);
    for (int a = 0; a < 4; ++a) ok = ok && std::isfinite(P.quat[a]);
    if (!ok) {
      if (out->bad_particles == 0) out->first_bad_particle = p;
      out->bad_particles += 1;
    }
  }
  if (out->bad_populations || out->bad_particles)
    return h->fail(MI_ESTATE, "non-finite state: " + std::to_string(out->bad_populations) +
                                  " populations at non-solid nodes (first at node " +
                                  std::to_string(out->first_bad_node) + "), " + std::to_string(out->bad_particles) +
                                  " particle states");
  return MI_OK;
}

static mi_status pop_copy(mi_delbm* h, const float* src_host, float* dst_host, size_t count) {
  if (!h) return MI_EINVAL;
  if (count != 19 * h->ncell) return h->fail(MI_EINVAL, "population count must be 19*nx*ny*nz");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  float* tmp = (float*)h->dalloc(count * sizeof(float));
  if (!tmp) return h->fail(MI_ENOMEM, "staging allocation failed");
  cudaError_t e;
  if (src_host) {
    e = cudaMemcpyAsync(tmp, src_host, count * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_pack(tmp, h->pop[h->cur], h->geom(), h->cfg.storage, h->stream);
  } else {
    e = launch_unpack(h->pop[h->cur], tmp, h->geom(), h->cfg.storage, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst_host, tmp, count * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  h->dfree(tmp);
  if (e != cudaSuccess) return h->cuda_fail(e, "population copy");
  return MI_OK;
}

mi_status mi_delbm_set_populations(mi_delbm* h, const float* host_f, size_t count) {
  if (!host_f) return h ? h->fail(MI_EINVAL, "null buffer") : MI_EINVAL;
  return pop_copy(h, host_f, nullptr, count);
}

mi_status mi_delbm_get_populations(mi_delbm* h, float* host_f, size_t count) {
  if (!host_f) return h ? h->fail(MI_EINVAL, "null buffer") : MI_EINVAL;
  return pop_copy(h, nullptr, host_f, count);
}

static mi_status raw_copy(mi_delbm* h, const void* src, void* dst, size_t bytes) {
  if (!h) return MI_EINVAL;
  if (bytes != 19 * h->ncell * h->esize) return h->fail(MI_EINVAL, "raw population bytes must be 19*ncell*element size");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  const size_t row = h->ncell * h->esize, pitch = h->plane * h->esize;
  cudaError_t e;
  if (src) e = cudaMemcpy2DAsync(h->pop[h->cur], pitch, src, row, row, 19, cudaMemcpyHostToDevice, h->stream);
  else e = cudaMemcpy2DAsync(dst, row, h->pop[h->cur], pitch, row, 19, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "raw population copy");
  return MI_OK;
}

mi_status mi_delbm_set_raw_populations(mi_delbm* h, const void* host, size_t bytes) {
  if (!host) return h ? h->fail(MI_EINVAL, "null buffer") : MI_EINVAL;
  return raw_copy(h, host, nullptr, bytes);
}

mi_status mi_delbm_get_raw_populations(mi_delbm* h, void* host, size_t bytes) {
  if (!host) return h ? h->fail(MI_EINVAL, "null buffer") : MI_EINVAL;
  return raw_copy(h, nullptr, host, bytes);
}

mi_status mi_delbm_get_device_view(mi_delbm* h, mi_delbm_device_view* v) {
  if (!h || !v) return MI_EINVAL;
  v->populations = h->pop[h->cur];
  v->plane_stride = h->plane;
  v->storage = h->cfg.storage;
  v->node_class = h->cls;
  v->owner = h->owner[h->owner_cur];
  v->stream = (void*)h->stream;
  return MI_OK;
}

mi_status mi_delbm_set_graphs(mi_delbm* h, int enable) {
  if (!h) return MI_EINVAL;
  if (enable < 0 || enable > 2) return h->fail(MI_EINVAL, "mi_delbm_set_graphs: mode must be 0, 1 or 2");
  h->use_graphs = enable != 0;
  h->loop_graphs = enable == 2;
  return MI_OK;
}

mi_status mi_delbm_set_guess(mi_delbm* h, int mode, const float* params) {
  if (!h) return MI_EINVAL;
  if (mode == MI_GUESS_PLAIN || mode == MI_GUESS_WARM) {
    if (h->learned || h->warm != (mode == MI_GUESS_WARM)) h->invalidate_graphs();
    h->learned = false;
    h->warm = mode == MI_GUESS_WARM;
    return MI_OK;
  }
  if (mode != MI_GUESS_LEARNED) return h->fail(MI_EINVAL, "set_guess: unknown mode");
  if (!params) return h->fail(MI_EINVAL, "set_guess: learned mode needs the MLP parameters");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  mi_status s = h->ensure_guess_buffers();
  if (s != MI_OK) return s;
  cudaError_t e = mlp_infer_prepare();
  if (e == cudaSuccess) e = mlp_tc_prepare();
  if (e == cudaSuccess) e = mlp_pack(params, h->mlp_image, h->stream);
  if (e == cudaSuccess)
    e = mlp_tc_pack(params, static_cast<unsigned char*>(h->mlp_image) + mlp_image_bytes(), h->stream);
  h->launches += 2;
  if (e != cudaSuccess) return h->cuda_fail(e, "set_guess: packing the parameters");
  h->invalidate_graphs();
  h->learned = true;
  h->warm = false;
  return MI_OK;
}

mi_status mi_delbm_pair_solve(mi_delbm* h, int n, const int* ij, const double* poses, int flags, const float* pred,
                              float* X, float* T, double* xm, int* iters, int* evals, int* status) {
  if (!h) return MI_EINVAL;
  const int known = MI_PAIR_FEATURES | MI_PAIR_PLAIN | MI_PAIR_LEARNED | MI_PAIR_LABELS | MI_PAIR_GUESS_ONLY;
  const bool plain = flags & MI_PAIR_PLAIN, lrn = flags & MI_PAIR_LEARNED;
  if (n < 0 || (flags & ~known) || (plain && lrn) || flags == 0)
    return h->fail(MI_EINVAL, "pair_solve: n < 0, unknown flags, or both PLAIN and LEARNED");
  if ((flags & MI_PAIR_GUESS_ONLY) && (!plain || (flags & MI_PAIR_LABELS)))
    return h->fail(MI_EINVAL, "pair_solve: GUESS_ONLY needs PLAIN and excludes LABELS");
  if ((flags & MI_PAIR_LABELS) && !plain && !lrn) return h->fail(MI_EINVAL, "pair_solve: LABELS needs a solve");
  if (n == 0) return MI_OK;
  if (!ij || !poses || ((flags & (MI_PAIR_FEATURES | MI_PAIR_LEARNED)) && !X) || (lrn && !pred) ||
      ((flags & MI_PAIR_LABELS) && !T) || ((plain || lrn) && (!xm || !iters || !evals || !status)))
    return h->fail(MI_EINVAL, "pair_solve: a required array is NULL");
  if (h->n_particles == 0) return h->fail(MI_EINVAL, "pair_solve: the handle has no particles (shapes)");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  mi_status s = h->ensure_particle_buffers();
  if (s != MI_OK) return s;
  PairSolveLaunch S;
  S.P = h->dP;
  S.np = h->n_particles;
  S.balls = h->dballs;
  S.n = n;
  S.ij = ij;
  S.poses = poses;
  S.flags = flags;
  S.pred = pred;
  S.X = X;
  S.T = T;
  S.xm = xm;
  S.iters = iters;
  S.evals = evals;
  S.status = status;
  cudaError_t e = launch_pair_solve(S, h->stream);
  h->launches += 1;
  if (e != cudaSuccess) return h->cuda_fail(e, "pair_solve: launch");
  return MI_OK;
}

mi_status mi_delbm_set_schedule(mi_delbm* h, int flags) {
  if (!h) return MI_EINVAL;
  if (flags & ~(MI_SCHEDULE_OVERLAP_BOUNDARY | MI_SCHEDULE_UNFUSED_DEM | MI_SCHEDULE_LINKS_BESIDE))
    return h->fail(MI_EINVAL, "mi_delbm_set_schedule: unknown flags");
  const bool ob = (flags & MI_SCHEDULE_OVERLAP_BOUNDARY) != 0, ud = (flags & MI_SCHEDULE_UNFUSED_DEM) != 0;
  const bool lb = (flags & MI_SCHEDULE_LINKS_BESIDE) != 0;
  if (h->overlap_boundary != ob || h->unfused_dem != ud || h->links_beside != lb) h->invalidate_graphs();
  h->overlap_boundary = ob;
  h->unfused_dem = ud;
  h->links_beside = lb;
  return MI_OK;
}

mi_status mi_delbm_set_momentum_rules(mi_delbm* h, int flags) {
  if (!h) return MI_EINVAL;
  if (flags & ~MI_MOMENTUM_COVER_UNCOVER) return h->fail(MI_EINVAL, "mi_delbm_set_momentum_rules: unknown flags");
  const bool cu = (flags & MI_MOMENTUM_COVER_UNCOVER) != 0;
  if (h->cover_uncover != cu) h->invalidate_graphs();
  h->cover_uncover = cu;
  return MI_OK;
}

mi_status mi_delbm_set_timing(mi_delbm* h, int enable) {
  if (!h) return MI_EINVAL;
  h->timing = enable != 0;
  return MI_OK;
}

mi_status mi_delbm_kernel_time(mi_delbm* h, const char* kernel, double* ms, long long* launches) {
  if (!h || !kernel || !ms || !launches) return MI_EINVAL;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_kernel_time");
  *ms = 0.0;
  *launches = 0;
  for (auto& t : h->timed) {
    float m = 0.f;
    if (t.kernel && std::strcmp(t.kernel, kernel) == 0 && cudaEventElapsedTime(&m, t.a, t.b) == cudaSuccess) {
      *ms += m;
      *launches += 1;
    }
  }
  return MI_OK;
}

mi_status mi_delbm_phase_times(mi_delbm* h, double ms[8], long long launches[8], int reset) {
  if (!h || !ms || !launches) return MI_EINVAL;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_phase_times");
  for (int b = 0; b < 8; ++b) {
    ms[b] = 0.0;
    launches[b] = 0;
  }
  for (auto& t : h->timed) {
    float m = 0.f;
    if (cudaEventElapsedTime(&m, t.a, t.b) == cudaSuccess) {
      ms[t.phase] += m;
      launches[t.phase] += 1;
    }
  }
  if (reset) {
    for (auto& t : h->timed) {
      h->event_pool.push_back(t.a);
      h->event_pool.push_back(t.b);
    }
    h->timed.clear();
  }
  return MI_OK;
}

long long mi_delbm_launch_count(const mi_delbm* h) { return h ? h->launches : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: launch shapes of the bulk and list kernels, measured with CUDA
// events and cached as one JSON object per line keyed by device and workload.
// ---------------------------------------------------------------------------
std::string mi_delbm::tune_key() const {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, cfg.device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, cfg.device);
  std::ostringstream k;
  k << "sm_" << major << minor << "/" << sm_count << "sm/" << cfg.nx << "x" << cfg.ny << "x" << cfg.nz << "/st"
    << cfg.storage << "/np" << n_particles << "/bb" << cfg.bb_mode << (forcing() ? "/force" : "");
  return k.str();
}

float mi_delbm::time_launches(int reps, const std::function<cudaError_t()>& fn) {
  cudaEvent_t a = event_from_pool(), b = event_from_pool();
  if (!a || !b) return -1.f;
  for (int i = 0; i < 2; ++i) fn();  // warm-up
  cudaEventRecord(a, stream);
  for (int i = 0; i < reps; ++i) fn();
  cudaEventRecord(b, stream);
  float ms = -1.f;
  if (cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  event_pool.push_back(a);
  event_pool.push_back(b);
  return ms / reps;
}

static bool read_cached(const char* path, const std::string& key, TuneChoice& t) {
  if (!path) return false;
  std::ifstream in(path);
  std::string line;
  const std::string tag = "\"key\": \"" + key + "\"";
  while (std::getline(in, line)) {
    if (line.find(tag) == std::string::npos) continue;
    auto grab = [&](const char* name, int& v) {
      const std::string n = std::string("\"") + name + "\": ";
      const size_t p = line.find(n);
      if (p == std::string::npos) return false;
      v = std::atoi(line.c_str() + p + n.size());
      return true;
    };
    int bx = 0, bl = 0, rows = 0, pairs = -1;
    if (grab("bulk_block_x", bx) && grab("list_blocks_per_sm", bl) && grab("bulk_rows", rows) &&
        grab("bulk_pairs", pairs) && bx > 0 && bx <= 256 && bx % 32 == 0 && bl > 0 && bl <= 64 &&
        (rows == 1 || rows == 2) && (pairs >= 0 && pairs <= 3)) {
      t.bulk_block_x = bx;
      t.list_blocks_per_sm = bl;
      t.bulk_rows = rows;
      t.bulk_pairs = pairs;
      return true;
    }
  }
  return false;
}

extern "C" mi_status mi_delbm_set_tuning(mi_delbm* h, int bulk_block_x, int bulk_rows, int bulk_pairs,
                                         int list_blocks_per_sm) {
  if (!h) return MI_EINVAL;
  if (bulk_block_x < 32 || bulk_block_x > 256 || bulk_block_x % 32 != 0 || (bulk_rows != 1 && bulk_rows != 2) ||
      bulk_pairs < 0 || bulk_pairs > 3 || (bulk_pairs && bulk_block_x > 128) || list_blocks_per_sm < 1 ||
      list_blocks_per_sm > 64)
    return h->fail(MI_EINVAL, "mi_delbm_set_tuning: block_x 32..256 (multiple of 32, <= 128 with pairs), rows 1|2, "
                              "pairs 0|1|2|3, list blocks per SM 1..64");
  h->tune.bulk_block_x = bulk_block_x;
  h->tune.bulk_rows = bulk_rows;
  h->tune.bulk_pairs = bulk_pairs;
  h->tune.list_blocks_per_sm = list_blocks_per_sm;
  h->invalidate_graphs();
  return MI_OK;
}

extern "C" mi_status mi_delbm_get_tuning(const mi_delbm* h, int* bulk_block_x, int* bulk_rows, int* bulk_pairs,
                                         int* list_blocks_per_sm) {
  if (!h) return MI_EINVAL;
  if (bulk_block_x) *bulk_block_x = h->tune.bulk_block_x;
  if (bulk_rows) *bulk_rows = h->tune.bulk_rows;
  if (bulk_pairs) *bulk_pairs = h->tune.bulk_pairs;
  if (list_blocks_per_sm) *list_blocks_per_sm = h->tune.list_blocks_per_sm;
  return MI_OK;
}

extern "C" mi_status mi_delbm_autotune(mi_delbm* h, const char* cache_path, int* bulk_block_x,
                                       int* list_blocks_per_sm) {
  if (!h) return MI_EINVAL;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  mi_status st = h->sync("mi_delbm_autotune");
  if (st != MI_OK) return st;
  const std::string key = h->tune_key();
  TuneChoice t = h->tune;
  if (!read_cached(cache_path, key, t)) {
    // bulk kernel: block width along x
    BulkLaunch L;
    L.A = h->pop[h->cur];
    L.B = h->pop[h->cur ^ 1];
    L.g = h->geom();
    L.p = h->collide_params();
    L.storage = h->cfg.storage;
    L.forcing = h->forcing();
    float best = 1e30f;
    // variants: 1 row, 2 rows, paired nodes (two register budgets for 16-bit
    // storages), four nodes per thread (16-bit storages)
    for (int variant = 0; variant < 5; ++variant) {
      const int pairs = variant >= 2 ? variant - 1 : 0;
      if (pairs && (h->cfg.nx % 2) != 0) continue;
      if (pairs >= 2 && h->cfg.storage == MI_STORE_F32) continue;
      if (pairs == 3 && (h->cfg.nx % 4) != 0) continue;
      for (int bx : {32, 64, 128, 256}) {
        const int span = pairs == 3 ? 4 * bx : pairs ? 2 * bx : bx;
        if (bx > 32 && span / 2 >= h->cfg.nx) break;
        if (pairs && bx > 128) break;
        L.block_x = bx;
        L.rows = variant == 1 ? 2 : 1;
        L.pairs = pairs != 0;
        L.pair_mode = pairs;
        const float ms = h->time_launches(5, [&] { return launch_bulk(L, h->stream); });
        if (ms > 0.f && ms < best) {
          best = ms;
          t.bulk_block_x = bx;
          t.bulk_rows = L.rows;
          t.bulk_pairs = pairs;
        }
      }
    }
    // list kernels: blocks per SM of the links' bounce-back and boundary-node
    // kernels, timed together (lists of the last step)
    if (h->n_particles > 0 && h->particles_ready) {
      DevCounters c;
      if (cudaMemcpy(&c, h->dctr, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess && c.n_bc > 0) {
        best = 1e30f;
        const TuneChoice keep = h->tune;
        for (int bl : {2, 4, 8, 16, 32}) {
          h->tune.list_blocks_per_sm = bl;
          BoundaryLaunch B = boundary_launch(h);
          const float ms = h->time_launches(5, [&] {
            const cudaError_t e = launch_links_ibb(B, h->stream);
            return e != cudaSuccess ? e : launch_boundary(B, h->stream);
          });
          if (ms > 0.f && ms < best) {
            best = ms;
            t.list_blocks_per_sm = bl;
          }
        }
        h->tune = keep;
        // the trial launches added into the force sums: clear them
        cudaMemsetAsync(h->facc, 0, sizeof(long long) * 6 * h->n_particles, h->stream);
      }
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_autotune");
    if (cache_path) {
      std::ofstream out(cache_path, std::ios::app);
      out << "{\"key\": \"" << key << "\", \"bulk_block_x\": " << t.bulk_block_x
          << ", \"bulk_rows\": " << t.bulk_rows << ", \"bulk_pairs\": " << t.bulk_pairs
          << ", \"list_blocks_per_sm\": " << t.list_blocks_per_sm << "}\n";
    }
  }
  t.tuned = true;
  h->tune = t;
  h->invalidate_graphs();
  if (bulk_block_x) *bulk_block_x = t.bulk_block_x;
  if (list_blocks_per_sm) *list_blocks_per_sm = t.list_blocks_per_sm;
  return MI_OK;
}

// ---------------------------------------------------------------------------
// Particles
// ---------------------------------------------------------------------------
namespace {
bool finite3(const double* v) { return v && std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

void rot_from_quat(const double q[4], double R[9]) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

bool invert3(const double A[9], double Ai[9]) {
  const double c0 = A[4] * A[8] - A[5] * A[7], c1 = A[5] * A[6] - A[3] * A[8], c2 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c0 + A[1] * c1 + A[2] * c2;
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
  const double id = 1.0 / det;
  Ai[0] = c0 * id; Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id; Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  Ai[3] = c1 * id; Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id; Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  Ai[6] = c2 * id; Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id; Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return true;
}
}  // namespace

extern "C" {

// Core-overlap test of a new particle (uploaded at slot id) against the
// existing ones: the plain closest-point solve between it and every particle
// whose bounding sphere it meets; overlap when the converged point lies
// inside a core (status 3).  Synchronises.
static mi_status overlap_check(mi_delbm* h, int id, const DevParticle& P) {
  std::vector<DevParticle> cur(id);
  cudaError_t e = cudaMemcpyAsync(cur.data(), h->dP, sizeof(DevParticle) * id, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "add_particle: reading particle states");
  std::vector<int> ij;
  std::vector<double> poses;
  for (int i = 0; i < id; ++i) {
    const double d0 = P.pos[0] - cur[i].pos[0], d1 = P.pos[1] - cur[i].pos[1], d2 = P.pos[2] - cur[i].pos[2];
    if (std::sqrt(d0 * d0 + d1 * d1 + d2 * d2) > P.Rb + cur[i].Rb) continue;
    ij.push_back(i);
    ij.push_back(id);
    for (int a = 0; a < 3; ++a) poses.push_back(cur[i].pos[a]);
    for (int a = 0; a < 4; ++a) poses.push_back(cur[i].quat[a]);
    for (int a = 0; a < 3; ++a) poses.push_back(P.pos[a]);
    for (int a = 0; a < 4; ++a) poses.push_back(P.quat[a]);
  }
  const int n = (int)(ij.size() / 2);
  if (n == 0) return MI_OK;
  int* d_ij = (int*)h->dalloc(sizeof(int) * 2 * n);
  double* d_pose = (double*)h->dalloc(sizeof(double) * 14 * n);
  double* d_xm = (double*)h->dalloc(sizeof(double) * 3 * n);
  int* d_out = (int*)h->dalloc(sizeof(int) * 3 * n);  // iterations, evaluations, status
  mi_status st = MI_OK;
  std::vector<int> status(n, 0);
  if (!d_ij || !d_pose || !d_xm || !d_out) {
    st = h->fail(MI_ENOMEM, "add_particle: overlap check buffers");
  } else {
    PairSolveLaunch S;
    std::memset(&S, 0, sizeof(S));
    S.P = h->dP;
    S.np = id + 1;
    S.balls = h->dballs;
    S.n = n;
    S.ij = d_ij;
    S.poses = d_pose;
    S.flags = MI_PAIR_PLAIN;
    S.xm = d_xm;
    S.iters = d_out;
    S.evals = d_out + n;
    S.status = d_out + 2 * n;
    e = cudaMemcpyAsync(d_ij, ij.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pose, poses.data(), sizeof(double) * 14 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_pair_solve(S, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), d_out + 2 * n, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->launches += 1;
    if (e != cudaSuccess) st = h->cuda_fail(e, "add_particle: overlap check");
  }
  h->dfree(d_ij);
  h->dfree(d_pose);
  h->dfree(d_xm);
  h->dfree(d_out);
  if (st != MI_OK) return st;
  for (int k = 0; k < n; ++k)
    if ((status[k] & 15) == 3)
      return h->fail(MI_EOVERLAP, "add_particle: the new particle's core overlaps particle " + std::to_string(ij[2 * k]));
  return MI_OK;
}

mi_status mi_delbm_add_particle(mi_delbm* h, int n, const double* centers, const double* k, double density,
                                double skin, const double pos[3], const double quat[4], const double vel[3],
                                const double omega[3], const mi_mass_props* mp, int* id_out) {
  if (!h) return MI_EINVAL;
  if (n < 1 || !centers || !k || !pos || !quat) return h->fail(MI_EINVAL, "add_particle: n_balls >= 1 and non-null centers, k, pos, quat required");
  if (!(density > 0.0) || !(skin >= 0.0) || !finite3(pos)) return h->fail(MI_EINVAL, "add_particle: density > 0, skin >= 0, finite pos required");
  const double qn2 = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
  if (!(qn2 > 0.0) || !std::isfinite(qn2)) return h->fail(MI_EINVAL, "add_particle: quaternion must be non-zero and finite");
  if ((vel && !finite3(vel)) || (omega && !finite3(omega))) return h->fail(MI_EINVAL, "add_particle: non-finite velocity");
  double sumk = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!(k[i] > 0.0) || !std::isfinite(k[i]) || !finite3(centers + 3 * i))
      return h->fail(MI_EINVAL, "add_particle: every k_i must be > 0 and every center finite");
    sumk += k[i];
  }
  const double re = std::sqrt(sumk);
  if (!(skin < re)) return h->fail(MI_EINVAL, "add_particle: skin radius must be below sqrt(sum k)");
  if (h->n_particles >= h->cfg.max_particles) return h->fail(MI_ECAPACITY, "add_particle: max_particles reached");
  if (h->n_balls_total + n > h->cfg.max_balls) return h->fail(MI_ECAPACITY, "add_particle: max_balls reached");
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  mi_status st = h->ensure_particle_buffers();
  if (st != MI_OK) return st;
  st = h->sync("add_particle");
  if (st != MI_OK) return st;

  std::vector<double> c(centers, centers + 3 * (size_t)n);
  const int off = h->n_balls_total;
  auto upload_balls = [&]() -> cudaError_t {
    std::vector<float4> bf(n), bs(2 * (size_t)n);
    std::vector<double> bd(4 * (size_t)n);
    for (int i = 0; i < n; ++i) {
      bf[i] = make_float4((float)c[3 * i], (float)c[3 * i + 1], (float)c[3 * i + 2], (float)k[i]);
      // hi + lo split for the wall-fraction kernel's float-float residual: a
      // centre coordinate below 1024 in magnitude as its nearest multiple of
      // 2^-12 (exact in FP32) plus the FP32 remainder, so that its difference
      // with a link origin split the same way is exact; k as its FP32 rounding
      // plus the remainder
      double hi[4];
      for (int a = 0; a < 3; ++a) {
        const double v = c[3 * i + a];
        hi[a] = std::fabs(v) < 1024.0 ? std::rint(v * 4096.0) / 4096.0 : (double)(float)v;
      }
      hi[3] = (double)(float)k[i];
      bs[2 * i] = make_float4((float)hi[0], (float)hi[1], (float)hi[2], (float)hi[3]);
      bs[2 * i + 1] = make_float4((float)(c[3 * i] - hi[0]), (float)(c[3 * i + 1] - hi[1]),
                                  (float)(c[3 * i + 2] - hi[2]), (float)(k[i] - hi[3]));
      bd[4 * i] = c[3 * i];
      bd[4 * i + 1] = c[3 * i + 1];
      bd[4 * i + 2] = c[3 * i + 2];
      bd[4 * i + 3] = k[i];
    }
    cudaError_t e = cudaMemcpyAsync(h->dballs + off, bf.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->dballs_d + 4 * (size_t)off, bd.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->dballs_s + 2 * (size_t)off, bs.data(), sizeof(float4) * 2 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e;
  };
  auto bounding = [&]() {
    double m = 0.0;
    for (int i = 0; i < n; ++i)
      m = std::fmax(m, std::sqrt(c[3 * i] * c[3 * i] + c[3 * i + 1] * c[3 * i + 1] + c[3 * i + 2] * c[3 * i + 2]));
    return m + re;
  };
  cudaError_t e = upload_balls();
  if (e != cudaSuccess) return h->cuda_fail(e, "add_particle: upload");

  double X[3] = {pos[0], pos[1], pos[2]};
  double R[9];
  rot_from_quat(quat, R);
  double mass, volume, I[9];
  if (!mp) {
    // midpoint quadrature of f >= 1, spacing 1/4, over [-Rb, Rb]^3
    const double hq = 0.25, Rb0 = bounding();
    const int nside = (int)std::ceil(2.0 * Rb0 / hq);
    const int blocks = h->sm_count * 4;
    double* part = (double*)h->dalloc(sizeof(double) * 10 * blocks);
    if (!part) return h->fail(MI_ENOMEM, "add_particle: quadrature buffer");
    e = launch_mass_quadrature(h->dballs + off, h->dballs_d + 4 * (size_t)off, n, Rb0, hq, nside, part, blocks, h->stream);
    std::vector<double> hpart(10 * (size_t)blocks);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hpart.data(), part, sizeof(double) * 10 * blocks, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->dfree(part);
    if (e != cudaSuccess) return h->cuda_fail(e, "add_particle: quadrature");
    double S[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < blocks; ++b)
      for (int j = 0; j < 10; ++j) S[j] += hpart[10 * (size_t)b + j];
    const double dv = hq * hq * hq;
    volume = S[0] * dv;
    if (!(volume > 0.0)) return h->fail(MI_EINVAL, "add_particle: the particle has no solid volume at spacing 1/4");
    const double cen[3] = {S[1] * dv / volume, S[2] * dv / volume, S[3] * dv / volume};
    double sec[9] = {S[4] * dv, S[5] * dv, S[6] * dv, S[5] * dv, S[7] * dv, S[8] * dv, S[6] * dv, S[8] * dv, S[9] * dv};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) sec[3 * a + b] -= volume * cen[a] * cen[b];
    const double tr = sec[0] + sec[4] + sec[8];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) I[3 * a + b] = density * ((a == b ? tr : 0.0) - sec[3 * a + b]);
    mass = density * volume;
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) c[3 * i + a] -= cen[a];
    for (int a = 0; a < 3; ++a) X[a] += R[3 * a] * cen[0] + R[3 * a + 1] * cen[1] + R[3 * a + 2] * cen[2];
    e = upload_balls();
    if (e != cudaSuccess) return h->cuda_fail(e, "add_particle: upload");
  } else {
    mass = mp->mass;
    volume = mp->volume;
    for (int j = 0; j < 9; ++j) I[j] = mp->inertia[j];
    if (!(mass > 0.0) || !(volume > 0.0)) return h->fail(MI_EINVAL, "add_particle: mass and volume must be > 0");
  }
  DevParticle P;
  std::memset(&P, 0, sizeof(P));
  if (!invert3(I, P.inv_inertia)) return h->fail(MI_EINVAL, "add_particle: singular inertia tensor");
  const double qn = std::sqrt(qn2);
  for (int a = 0; a < 3; ++a) {
    P.pos[a] = X[a];
    P.vel[a] = vel ? vel[a] : 0.0;
    P.omega[a] = omega ? omega[a] : 0.0;
  }
  (void)qn;  // kept as given: the kernels normalise with the same operations as the definition
  for (int j = 0; j < 4; ++j) P.quat[j] = quat[j];
  for (int j = 0; j < 9; ++j) P.inertia[j] = I[j];
  P.mass = mass;
  P.volume = volume;
  P.density = density;
  P.skin = skin;
  P.re = re;
  P.core_s = (float)(((re - skin) / re) * ((re - skin) / re));
  P.re_f = (float)re;
  P.skin_f = (float)skin;
  P.Rb = bounding();
  P.Rb_f = (float)P.Rb;
  {
    // tight radius: for |x| > max|c_i|, f(x) <= sum k_i / (|x| - |c_i|)^2, which decreases
    // in |x|; beyond its root Rt (<= Rb) every node is fluid
    double cmax = 0.0;
    std::vector<double> cn(n);
    for (int i = 0; i < n; ++i) {
      cn[i] = std::sqrt(c[3 * i] * c[3 * i] + c[3 * i + 1] * c[3 * i + 1] + c[3 * i + 2] * c[3 * i + 2]);
      cmax = std::fmax(cmax, cn[i]);
    }
    double lo = cmax, hi = P.Rb;
    for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
      const double mid = 0.5 * (lo + hi);
      double sum = 0.0;
      for (int i = 0; i < n; ++i) sum += k[i] / ((mid - cn[i]) * (mid - cn[i]));
      if (sum > 1.0) lo = mid;
      else hi = mid;
    }
    P.Rt = std::fmin(hi * (1.0 + 1e-9) + 1e-9, P.Rb);
  }
  P.ball_off = off;
  P.n_balls = n;
  for (int a = 0; a < 3; ++a) {
    P.ext[a] = (int)std::ceil(2.0 * P.Rt) + 4;
    P.lo[a] = BOX_NONE;
    P.lo_hist[0][a] = BOX_NONE;
    P.lo_hist[1][a] = BOX_NONE;
  }
  const int id = h->n_particles;
  e = cudaMemcpyAsync(h->dP + id, &P, sizeof(P), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "add_particle: particle upload");
  if (h->cfg.check_overlap && id > 0) {
    // nothing is committed yet: on rejection the slot and the ball range are reused by the next add
    if ((st = overlap_check(h, id, P)) != MI_OK) return st;
  }
  h->hp.push_back(P);
  for (int i = 0; i < n; ++i) {
    h->hballs.push_back(make_float4((float)c[3 * i], (float)c[3 * i + 1], (float)c[3 * i + 2], (float)k[i]));
    for (int a = 0; a < 3; ++a) h->hballs_d.push_back(c[3 * i + a]);
    h->hballs_d.push_back(k[i]);
  }
  h->n_balls_total += n;
  if (n > h->max_balls_pp) h->max_balls_pp = n;
  h->n_particles += 1;
  // list capacities and box-kernel grid from the particles' box extents
  unsigned long long sbc = 0;
  for (const auto& q : h->hp) {
    const unsigned long long e2 = (unsigned long long)(q.ext[0] + 4) * (q.ext[0] + 4);
    sbc += 6ull * e2;
  }
  if (sbc > 0x3FFFFFFFull) sbc = 0x3FFFFFFFull;
  st = h->ensure_list_capacity((unsigned)sbc, (unsigned)std::min<unsigned long long>(6ull * sbc, 0xFFFFFFF0ull), (unsigned)sbc);
  if (st != MI_OK) return st;
  // box-kernel blocks per particle: about 8192 box nodes per flag block, and
  // 8 warps of about 64 rows each per classification block (the classified
  // region, old and new box widened by 2, has fewer than (ext + 8)^2 rows).
  // Few long-lived blocks: these kernels run beside the bulk kernel, and the
  // fewer SM slots they hold at a time, the less they slow it (eight times
  // more blocks made the settling-tank step 2.4 % slower; sixteen times
  // fewer made the particle chain outlast the 16-bit bulk kernel)
  const int npart = h->n_particles, stride = h->cfg.max_particles + 1;
  std::vector<int> boff(2 * (size_t)stride, 0);
  for (int q = 0; q < npart; ++q) {
    const int* e = h->hp[q].ext;
    const long long fb = ((long long)e[0] * e[1] * e[2] + 8191) / 8192;
    const long long cb = ((long long)(e[1] + 8) * (e[2] + 8) + 511) / 512;
    boff[q + 1] = boff[q] + (int)std::min<long long>(std::max<long long>(fb, 1), 8192);
    boff[stride + q + 1] = boff[stride + q] + (int)std::min<long long>(std::max<long long>(cb, 1), 4096);
  }
  h->flag_blocks = std::max(boff[npart], 1);
  h->classify_blocks = std::max(boff[stride + npart], 1);
  cudaError_t ce = cudaMemcpyAsync(h->dblk_off, boff.data(), sizeof(int) * boff.size(), cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return h->cuda_fail(ce, "mi_delbm_add_particle: block offsets");
  h->invalidate_graphs();
  if (id_out) *id_out = id;
  return MI_OK;
}

int mi_delbm_num_particles(const mi_delbm* h) { return h ? h->n_particles : 0; }

mi_status mi_delbm_get_particle_state(mi_delbm* h, int id, double pos[3], double quat[4], double vel[3],
                                      double omega[3]) {
  if (!h) return MI_EINVAL;
  if (id < 0 || id >= h->n_particles) return h->fail(MI_EINVAL, "get_particle_state: bad id");
  mi_status st = h->sync("get_particle_state");
  if (st != MI_OK) return st;
  DevParticle& P = h->hp[id];
  cudaError_t e = cudaMemcpy(&P, h->dP + id, sizeof(P), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_particle_state");
  for (int a = 0; a < 3; ++a) {
    if (pos) pos[a] = P.pos[a];
    if (vel) vel[a] = P.vel[a];
    if (omega) omega[a] = P.omega[a];
  }
  if (quat)
    for (int j = 0; j < 4; ++j) quat[j] = P.quat[j];
  return MI_OK;
}

mi_status mi_delbm_set_particle_state(mi_delbm* h, int id, const double pos[3], const double quat[4],
                                      const double vel[3], const double omega[3]) {
  if (!h) return MI_EINVAL;
  if (id < 0 || id >= h->n_particles) return h->fail(MI_EINVAL, "set_particle_state: bad id");
  if ((pos && !finite3(pos)) || (vel && !finite3(vel)) || (omega && !finite3(omega)))
    return h->fail(MI_EINVAL, "set_particle_state: non-finite value");
  mi_status st = h->sync("set_particle_state");
  if (st != MI_OK) return st;
  DevParticle& P = h->hp[id];
  cudaError_t e = cudaMemcpy(&P, h->dP + id, sizeof(P), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "set_particle_state");
  if (quat) {
    const double qn = std::sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    if (!(qn > 0.0) || !std::isfinite(qn)) return h->fail(MI_EINVAL, "set_particle_state: bad quaternion");
    for (int j = 0; j < 4; ++j) P.quat[j] = quat[j];
  }
  for (int a = 0; a < 3; ++a) {
    if (pos) P.pos[a] = pos[a];
    if (vel) P.vel[a] = vel[a];
    if (omega) P.omega[a] = omega[a];
  }
  e = cudaMemcpy(h->dP + id, &P, sizeof(P), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return h->cuda_fail(e, "set_particle_state");
  return MI_OK;
}

mi_status mi_delbm_set_particle_states(mi_delbm* h, const double* states, int n) {
  if (!h || !states) return MI_EINVAL;
  if (n != h->n_particles) return h->fail(MI_EINVAL, "set_particle_states: n must equal the particle count");
  if (n == 0) return MI_OK;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  static_assert(offsetof(DevParticle, pos) == 0 && offsetof(DevParticle, omega) == 10 * sizeof(double),
                "kinematic fields must lead DevParticle");
  cudaError_t e = cudaMemcpy2DAsync(h->dP, sizeof(DevParticle), states, 13 * sizeof(double), 13 * sizeof(double),
                                    (size_t)n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "set_particle_states");
  return MI_OK;
}

mi_status mi_delbm_get_particle_states(mi_delbm* h, double* states, int n) {
  if (!h || !states) return MI_EINVAL;
  if (n != h->n_particles) return h->fail(MI_EINVAL, "get_particle_states: n must equal the particle count");
  if (n == 0) return MI_OK;
  if (!h->set_device()) return h->fail(MI_ECUDA, "cudaSetDevice failed");
  cudaError_t e = cudaMemcpy2DAsync(states, 13 * sizeof(double), h->dP, sizeof(DevParticle), 13 * sizeof(double),
                                    (size_t)n, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_particle_states");
  return MI_OK;
}

mi_status mi_delbm_get_particle_shape(mi_delbm* h, int id, double* centers, double* k, int cap, int* n_out,
                                      mi_mass_props* mp, double* Rb) {
  if (!h) return MI_EINVAL;
  if (id < 0 || id >= h->n_particles) return h->fail(MI_EINVAL, "get_particle_shape: bad id");
  const DevParticle& P = h->hp[id];
  if (n_out) *n_out = P.n_balls;
  if ((centers || k) && cap < P.n_balls) return h->fail(MI_ECAPACITY, "get_particle_shape: cap below the ball count");
  for (int i = 0; i < P.n_balls; ++i) {
    const double* b = &h->hballs_d[4 * (size_t)(P.ball_off + i)];
    if (centers)
      for (int a = 0; a < 3; ++a) centers[3 * i + a] = b[a];
    if (k) k[i] = b[3];
  }
  if (mp) {
    mp->mass = P.mass;
    mp->volume = P.volume;
    for (int j = 0; j < 9; ++j) mp->inertia[j] = P.inertia[j];
  }
  if (Rb) *Rb = P.Rb;
  return MI_OK;
}

mi_status mi_delbm_forces(mi_delbm* h, double* F_hydro, double* T_hydro, double* F_contact, double* T_contact) {
  if (!h) return MI_EINVAL;
  mi_status st = h->sync("mi_delbm_forces");
  if (st != MI_OK) return st;
  const int np = h->n_particles;
  if (np == 0) return MI_OK;
  std::vector<long long> fa(6 * (size_t)np), fcl(6 * (size_t)np);
  cudaError_t e = cudaMemcpy(fa.data(), h->facc, sizeof(long long) * 6 * np, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(fcl.data(), h->fc, sizeof(long long) * 6 * np, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_forces");
  for (int p = 0; p < np; ++p)
    for (int a = 0; a < 3; ++a) {
      if (F_hydro) F_hydro[3 * p + a] = (double)fa[6 * p + a] * FIX_INV;
      if (T_hydro) T_hydro[3 * p + a] = (double)fa[6 * p + 3 + a] * FIX_INV;
      if (F_contact) F_contact[3 * p + a] = (double)fcl[6 * p + a] * FIX_INV;
      if (T_contact) T_contact[3 * p + a] = (double)fcl[6 * p + 3 + a] * FIX_INV;
    }
  return h->check_status(false);
}

mi_status mi_delbm_get_node_classes(mi_delbm* h, uint8_t* node_class, uint32_t* owner, size_t count) {
  if (!h) return MI_EINVAL;
  if (count != h->ncell) return h->fail(MI_EINVAL, "get_node_classes: count must be nx*ny*nz");
  mi_status st = h->sync("get_node_classes");
  if (st != MI_OK) return st;
  cudaError_t e = cudaSuccess;
  if (node_class) e = cudaMemcpy(node_class, h->cls, h->ncell, cudaMemcpyDeviceToHost);
  if (owner && e == cudaSuccess) {
    if (h->particles_ready) e = cudaMemcpy(owner, h->owner[h->owner_cur], 4 * h->ncell, cudaMemcpyDeviceToHost);
    else std::memset(owner, 0xFF, 4 * h->ncell);
  }
  if (e != cudaSuccess) return h->cuda_fail(e, "get_node_classes");
  return MI_OK;
}

mi_status mi_delbm_get_links(mi_delbm* h, size_t cap, int32_t* cell, int8_t* dir, int32_t* particle, float* q,
                             size_t* n_out) {
  if (!h || !n_out) return MI_EINVAL;
  mi_status st = h->sync("get_links");
  if (st != MI_OK) return st;
  *n_out = 0;
  if (!h->particles_ready) return MI_OK;
  DevCounters c;
  cudaError_t e = cudaMemcpy(&c, h->dctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_links");
  const size_t nl = std::min<size_t>(c.n_links, h->cap_links), nb = std::min<size_t>(c.n_bc, h->cap_bc);
  *n_out = nl;
  if (nl > cap) return h->fail(MI_ECAPACITY, "get_links: cap below the link count");
  std::vector<uint32_t> lbc(nl), lp(nl), bcc(nb);
  std::vector<uint8_t> ld(nl);
  std::vector<float> lq(nl);
  if (nl) {
    e = cudaMemcpy(lbc.data(), h->link_bc, 4 * nl, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lp.data(), h->link_p, 4 * nl, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ld.data(), h->link_dir, nl, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lq.data(), h->link_q, 4 * nl, cudaMemcpyDeviceToHost);
  }
  if (nb && e == cudaSuccess) e = cudaMemcpy(bcc.data(), h->bc_cell, 4 * nb, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_links");
  for (size_t l = 0; l < nl; ++l) {
    if (cell) cell[l] = lbc[l] < nb ? (int32_t)bcc[lbc[l]] : -1;
    if (dir) dir[l] = (int8_t)ld[l];
    if (particle) particle[l] = (int32_t)lp[l];
    if (q) q[l] = lq[l];
  }
  return MI_OK;
}


mi_status mi_delbm_contacts(mi_delbm* h, mi_contact* out, int cap, int* n_out) {
  if (!h || !n_out) return MI_EINVAL;
  mi_status st = h->sync("mi_delbm_contacts");
  if (st != MI_OK) return st;
  *n_out = 0;
  if (!h->contacts_ready) return MI_OK;
  DevCounters c;
  cudaError_t e = cudaMemcpy(&c, h->dctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_contacts");
  const unsigned n = std::min(c.n_pairs, h->cap_items);
  *n_out = (int)n;
  if ((int)n > cap || (n > 0 && !out)) return h->fail(MI_ECAPACITY, "mi_delbm_contacts: cap below the candidate count");
  if (n) {
    // the device keeps compact records (FP32 geometry relative to the origin
    // of particle i); the world contact point is formed here in FP64
    std::vector<ContactRec> tmp(n);
    e = cudaMemcpy(tmp.data(), h->recs, sizeof(ContactRec) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return h->cuda_fail(e, "mi_delbm_contacts");
    for (unsigned k = 0; k < n; ++k) {
      const ContactRec& r = tmp[k];
      mi_contact& c = out[k];
      c.i = r.i;
      c.j = r.j;
      for (int a = 0; a < 3; ++a) {
        c.xcp[a] = r.X[a] + (double)r.r[a];
        c.n[a] = (double)r.n[a];
      }
      c.delta = (double)r.delta;
      c.iters = r.iters;
      c.status = r.status;
    }
  }
  return h->check_status(false);
}

mi_status mi_delbm_get_stats(mi_delbm* h, mi_delbm_stats* out) {
  if (!h || !out) return MI_EINVAL;
  std::memset(out, 0, sizeof(*out));
  mi_status st = h->sync("get_stats");
  if (st != MI_OK) return st;
  if (!h->particles_ready) return MI_OK;
  DevCounters c;
  cudaError_t e = cudaMemcpy(&c, h->dctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_stats");
  out->boundary_nodes = c.n_bc;
  out->links = c.n_links;
  out->new_nodes = c.n_new;
  out->candidate_pairs = c.n_pairs;
  out->contacts = c.n_contacts;
  out->status = c.status;
  unsigned zero = 0;
  e = cudaMemcpy(&h->dctr->status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return h->cuda_fail(e, "get_stats");
  return MI_OK;
}

}  // extern "C"
