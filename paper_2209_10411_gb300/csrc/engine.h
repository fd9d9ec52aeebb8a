// Handle state of libmi_delbm (internal; the C-ABI is include/mi_delbm.h).
#pragma once

#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "mi_internal.cuh"

struct TimedLaunch {
  int phase;
  cudaEvent_t a, b;
  const char* kernel;  // the kernel's name (a string literal), for mi_delbm_kernel_time
};

struct TuneChoice {
  int bulk_block_x = 128;     // threads per block of the bulk kernel (along x)
  int bulk_rows = 1;          // rows per thread of the bulk kernel
  int bulk_pairs = 0;         // 0 one node per thread; 1, 2: two x-adjacent nodes per thread with paired
                              // accesses (nx even; for 16-bit storages 1 and 2 select the register budget)
  int list_blocks_per_sm = 8; // grid of the list kernels (links, refill, boundary, near) per SM
  bool tuned = false;
};

struct mi_delbm {
  mi_delbm_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // side branches of a step (high priority; joined before the step ends):
  // 0 wall fractions, 1 first-substep contacts, 2 particle chain
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork[3] = {nullptr, nullptr, nullptr}, ev_join[3] = {nullptr, nullptr, nullptr};
  // CUDA graphs of one step, keyed by (population buffer, owner buffer) parity
  bool use_graphs = true;
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  long long glaunches[4] = {0, 0, 0, 0};
  // device-loop graphs (mi_delbm_set_graphs(h, 2)): a conditional while node
  // whose body is two whole steps, keyed like gexec; loop_count is the
  // device counter of step pairs left
  bool loop_graphs = false;
  cudaGraphExec_t gloop[4] = {nullptr, nullptr, nullptr, nullptr};
  long long gloop_launches[4] = {0, 0, 0, 0};
  int* loop_count = nullptr;

  size_t ncell = 0;   // nx*ny*nz
  size_t plane = 0;   // elements between population planes
  size_t esize = 4;   // bytes per stored population element

  void* pop[2] = {nullptr, nullptr};  // pop[cur] holds f+(t)
  int cur = 0;
  uint8_t* cls = nullptr;             // node classes
  uint32_t* owner[2] = {nullptr, nullptr};
  int owner_cur = 0;

  int n_particles = 0;
  long long step_index = 0;
  int sm_count = 148;

  // particles (allocated at the first add_particle)
  bool particles_ready = false;
  std::vector<mi::DevParticle> hp;   // host mirror (pose fields refreshed on demand)
  std::vector<float4> hballs;
  std::vector<double> hballs_d;
  mi::DevParticle* dP = nullptr;
  float4* dballs = nullptr;
  double* dballs_d = nullptr;
  float4* dballs_s = nullptr;   // per ball: FP32 (c, k), then the FP32 remainders of the FP64 (c, k)
  int n_balls_total = 0;
  int max_balls_pp = 0;              // largest ball count of one particle
  uint32_t* stamp = nullptr;
  mi::DevCounters* dctr = nullptr;
  long long* facc = nullptr;         // np x 6 fixed point (hydrodynamic)
  long long* fc = nullptr;           // np x 6 fixed point (contact)
  // contacts (allocated at the first contact phase)
  bool contacts_ready = false;
  int* item_i = nullptr;
  int* item_j = nullptr;
  unsigned cap_items = 0;
  mi::ContactRec* recs = nullptr;
  mi::HistEntry* hist_pair = nullptr;
  mi::HistEntry* hist_wall = nullptr;
  unsigned* work = nullptr;
  long long* substep = nullptr;
  float4* bp_pos = nullptr;           // FP32 positions and radii of the broad phase
  float4* bp_quat = nullptr;          // FP32 unit quaternions of the substep
  float4* bp_lo = nullptr;            // FP32 position remainders of the substep
  float4* bp_vel = nullptr;           // FP32 velocities and angular velocities of the substep (2 per particle)
  // learned contact guess (MI_GUESS_LEARNED): parameters and per-item buffers
  bool learned = false;
  unsigned guess_wait_limit = 0;     // try_wait rounds of the tcgen05 MLP kernel's waits (0: its default)
  int guess_stall = 0;               // fault-injection tests: the MLP kernel first waits on a barrier nothing arrives at
  long long* check_buf = nullptr;    // mi_delbm_check: count of non-finite values and the first node
  bool warm = false;                 // MI_GUESS_WARM
  void* mlp_image = nullptr;         // packed BF16 parameters of the fused inference kernel
  float* guess_feat = nullptr;       // cap_items x 64
  float* guess_pred = nullptr;       // cap_items x 4
  // lists
  uint32_t *bc_cell = nullptr, *bc_mask = nullptr, *bc_loff = nullptr;
  uint32_t *link_bc = nullptr, *link_p = nullptr;
  uint8_t* link_dir = nullptr;
  float* link_q = nullptr;
  float* link_g = nullptr;
  long long* ibb_part = nullptr;     // per-block momentum-exchange sums of the link kernel
  uint32_t* new_cell = nullptr;
  uint32_t* cov_cell = nullptr;     // nodes covered this step (cover/uncover rule; capacity cap_new)
  unsigned cap_bc = 0, cap_links = 0, cap_new = 0;
  // list sizes a step that overflowed needed: the lists grow to them before the next step
  unsigned need_bc = 0, need_links = 0, need_new = 0;
  void* bc_tmp = nullptr;            // 19 stored values per boundary node (overlapped schedule)
  bool overlap_boundary = false;     // boundary nodes computed beside the bulk kernel, scattered after it
  bool links_beside = false;         // the links' bounce-back beside the bulk kernel
  bool unfused_dem = false;          // DEM substeps as separate launches even where the fused kernel applies
  bool cover_uncover = false;        // covered/uncovered-node momentum joins the hydrodynamic sums
  // blocks of the box kernels, sized per particle: device offsets (particle
  // p owns blocks [off[p], off[p + 1])) of the flag and clear kernels, then of
  // the classification, max_particles + 1 each; the totals are the grids
  int* dblk_off = nullptr;
  int flag_blocks = 1, classify_blocks = 1;

  TuneChoice tune;

  bool timing = false;
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  long long launches = 0;

  std::vector<std::pair<void*, size_t>> allocs;
  std::string err;

  mi_status fail(mi_status s, const std::string& msg);
  mi_status cuda_fail(cudaError_t e, const char* what);
  void* dalloc(size_t bytes);
  void dfree(void* p);
  cudaEvent_t event_from_pool();
  bool set_device();
  mi::LatticeGeom geom() const;
  mi::CollideParams collide_params() const;
  bool forcing() const;

  mi_status grow_lists_if_needed();
  mi_status loop_steps(long long pairs);
  mi_status run_phases(unsigned phases);
  mi_status phase_flag(cudaStream_t st);
  mi_status phase_links(cudaStream_t st);
  mi_status phase_refill(cudaStream_t st);
  mi_status phase_near();
  mi_status phase_bulk();
  mi_status phase_links_ibb(cudaStream_t st);
  mi_status phase_boundary();
  mi_status phase_boundary_beside(cudaStream_t st);
  mi_status phase_scatter_boundary();
  mi_status phase_swap();
  mi_status phase_dem_fused();
  mi_status phase_integrate(bool with_contacts);
  mi_status phase_contact(cudaStream_t st);
  mi_status graph_step();
  std::string tune_key() const;
  float time_launches(int reps, const std::function<cudaError_t()>& fn);
  void invalidate_graphs();
  mi_status fork(cudaStream_t from, cudaStream_t to, int slot);
  mi_status join_record(cudaStream_t from, int slot);
  mi_status join_wait(int slot);
  mi_status ensure_contact_buffers();
  mi_status ensure_guess_buffers();

  mi_status ensure_particle_buffers();
  mi_status ensure_list_capacity(unsigned bc, unsigned links, unsigned nnew);
  mi::ParticleLaunch particle_launch() const;
  mi_status check_status(bool clear);
  mi_status sync(const char* what);
};
