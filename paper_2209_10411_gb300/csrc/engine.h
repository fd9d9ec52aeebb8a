// Handle state of libmi_delbm (internal; the C-ABI is include/mi_delbm.h).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "mi_internal.cuh"

struct TimedLaunch {
  int phase;
  cudaEvent_t a, b;
};

struct TuneChoice {
  int bulk_block_x = 128;
};

struct mi_delbm {
  mi_delbm_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;

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

  mi_status run_phases(unsigned phases);
  mi_status phase_bulk();
  mi_status phase_swap();
};
