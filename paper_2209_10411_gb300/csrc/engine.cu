// Engine and C-ABI of libmi_delbm: owns the device state of one lattice and
// its particles, sequences the kernels of one coupled step on one stream.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

using namespace mi;

namespace {
thread_local std::string g_create_error;

// Kernel-launch helper: runs `fn` (which returns a cudaError_t) as one launch
// of `phase`, bracketed by timing events when timing is enabled.
template <class F>
mi_status launch_phase(mi_delbm* h, unsigned phase_bit, F&& fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = h->event_from_pool();
    b = h->event_from_pool();
    if (!a || !b) return h->fail(MI_ECUDA, "cudaEventCreate failed");
    cudaEventRecord(a, h->stream);
  }
  cudaError_t e = fn();
  h->launches += 1;
  if (e != cudaSuccess) return h->fail(MI_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  if (h->timing) {
    cudaEventRecord(b, h->stream);
    int idx = 0;
    while ((1u << idx) != phase_bit && idx < 7) ++idx;
    h->timed.push_back({idx, a, b});
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
mi_status mi_delbm::phase_bulk() {
  BulkLaunch L;
  L.A = pop[cur];
  L.B = pop[cur ^ 1];
  L.cls = n_particles > 0 ? cls : nullptr;
  L.g = geom();
  L.p = collide_params();
  L.storage = cfg.storage;
  L.forcing = forcing();
  L.block_x = tune.bulk_block_x;
  return launch_phase(this, MI_PHASE_BULK, [&] { return launch_bulk(L, stream); });
}

mi_status mi_delbm::phase_swap() {
  cur ^= 1;
  step_index += 1;
  return MI_OK;
}

mi_status mi_delbm::run_phases(unsigned phases) {
  mi_status s = MI_OK;
  if ((phases & MI_PHASE_BULK) && (s = phase_bulk()) != MI_OK) return s;
  if ((phases & MI_PHASE_SWAP) && (s = phase_swap()) != MI_OK) return s;
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
  if (cfg->dem_substeps < 1 || cfg->max_particles < 0 || cfg->max_balls < 0) {
    g_create_error = "mi_delbm_create: dem_substeps must be >= 1 and capacities >= 0";
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
  h->tune.bulk_block_x = cfg->nx >= 128 ? 128 : (cfg->nx >= 64 ? 64 : 32);
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
  for (int n = 0; n < n_steps; ++n) {
    mi_status s = h->run_phases(MI_PHASE_ALL);
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
  return h->run_phases(phases);
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

mi_status mi_delbm_set_timing(mi_delbm* h, int enable) {
  if (!h) return MI_EINVAL;
  h->timing = enable != 0;
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
