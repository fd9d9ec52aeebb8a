/*
 * mi_delbm.h -- C-ABI of the GB300 (sm_103a) per-timestep fluid-particle step
 * of the Metaball-Imaging Discrete Element Lattice Boltzmann Method
 * (Zhang et al., arXiv 2209.10411).
 *
 * One handle owns one lattice and its particles on one GPU.  The step it runs
 * is, in this order (the paper's Sec. 2.3 describes the parts, not the order;
 * this order is the library's reading):
 *
 *   1. solid flagging of lattice nodes from each particle's metaball field
 *      f(x) = sum_i k_i / |x - c_i|^2 >= 1 in the particle's body frame
 *      (Sec. 2.1, Eq. 1; node classes fluid / solid / boundary, Sec. 2.3.2);
 *   2. boundary links (fluid node -> solid neighbour) and the wall fraction q
 *      solving f(x_f + q e_i) = 1 along the link (Sec. 2.3.2);
 *   3. local bounce-back refill of nodes a particle has just uncovered
 *      (Sec. 2.3.2, refill equation);
 *   4. fused D3Q19 BGK pull stream-collide of every bulk fluid node;
 *   5. interpolated bounce-back on every boundary link (Sec. 2.3.2, Eqs. of
 *      the IBB rule and the u_d interpolation), collision of boundary nodes,
 *      and the Galilean-invariant momentum exchange summed to per-particle
 *      hydrodynamic force and torque;
 *   6. DEM: broad phase, Newton-Raphson closest points between sphero-metaball
 *      particles and between particles and walls, linear spring-dashpot
 *      forces (Sec. 2.3.1, Eqs. CM_coreF, grad, cp, contactprop, metawallcp,
 *      contactprop2);
 *   7. rigid-body update (Sec. 2.3.1, Newton-Euler equations).
 *
 * Conventions (all calls):
 *   - Lattice units: dx = dt = 1, C = 1, c_s^2 = 1/3.  Node (i, j, k) sits at
 *     position (i, j, k).  Populations are addressed [q][z][y][x] with x
 *     fastest; q follows the D3Q19 order 0 = rest, 1..6 = +x,-x,+y,-y,+z,-z,
 *     7..18 = (+x+y),(-x-y),(+x-y),(-x+y),(+x+z),(-x-z),(+x-z),(-x+z),
 *     (+y+z),(-y-z),(+y-z),(-y+z).
 *   - Every call returns mi_status; MI_OK is 0.  On failure a message is kept
 *     and mi_delbm_last_error() returns it.  No call aborts the process.
 *   - Host buffers passed in are copied; the caller keeps ownership.  Output
 *     buffers are caller-allocated.
 *   - A handle is not thread-safe: use it from one host thread.  All device
 *     work of a handle runs in order on its stream.  mi_delbm_step is
 *     asynchronous; the query calls synchronise the stream.
 *   - A device-side failure of the method (Newton not converged, a list over
 *     capacity) never traps the GPU: it is recorded in device status words and
 *     reported by the next synchronising call.
 */
#ifndef MI_DELBM_H
#define MI_DELBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MI_DELBM_ABI_VERSION 2

typedef enum {
  MI_OK = 0,
  MI_EINVAL = 1,     /* an argument is out of range or inconsistent            */
  MI_ENOMEM = 2,     /* a device or host allocation failed                      */
  MI_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error) */
  MI_ECAPACITY = 4,  /* an output buffer or an internal list is too small       */
  MI_EOVERLAP = 5,   /* a new particle's core overlaps an existing particle     */
  MI_ESTATE = 6,     /* the call is not valid in the handle's current state     */
  MI_ETIMEOUT = 7,   /* a bounded device wait gave up                           */
  MI_ENOTSUP = 8     /* the option is not supported by this build               */
} mi_status;

/* Population storage in HBM (the arithmetic is FP32 in every mode). */
enum {
  MI_STORE_F32 = 0,      /* f_i as float                                       */
  MI_STORE_F16_DEV = 1,  /* f_i - w_i as IEEE half, round to nearest even      */
  MI_STORE_BF16_DEV = 2  /* f_i - w_i as bfloat16, round to nearest even       */
};

/* Particle-wall link rule. */
enum {
  MI_BB_IBB = 0,   /* the paper's interpolated bounce-back (Sec. 2.3.2)      */
  MI_BB_LADD = 1   /* halfway bounce-back with the moving-wall term (q = 1/2) */
};

/* Newton initial guess for contact detection. */
enum {
  MI_GUESS_PLAIN = 0,   /* midpoint of the closest pair of control points     */
  MI_GUESS_LEARNED = 1, /* the loaded MLP proposes the guess and active subset */
  MI_GUESS_WARM = 2     /* the pair's closest point of the previous DEM substep
                           (when the pair was solved there), else the plain guess */
};

/* Step phases, for mi_delbm_step_phases (tests and profiling). */
enum {
  MI_PHASE_FLAG = 1u << 0,      /* solid flags, node classes, boundary/new lists */
  MI_PHASE_LINKS = 1u << 1,     /* wall fraction q of every boundary link        */
  MI_PHASE_REFILL = 1u << 2,    /* populations of newly uncovered nodes          */
  MI_PHASE_BULK = 1u << 3,      /* stream-collide of bulk fluid nodes            */
  MI_PHASE_BOUNDARY = 1u << 4,  /* IBB + collide of boundary nodes, momentum exchange */
  MI_PHASE_SWAP = 1u << 5,      /* population buffers swap, flag history advances */
  MI_PHASE_CONTACT = 1u << 6,   /* broad phase, Newton contacts, contact forces  */
  MI_PHASE_INTEGRATE = 1u << 7, /* rigid-body update                             */
  MI_PHASE_ALL = 0xFFu
};

typedef struct mi_delbm_config {
  int nx, ny, nz;                /* lattice nodes per axis, each >= 1           */
  double tau;                    /* BGK relaxation time, > 1/2                  */
  double rho0;                   /* reference density (1 in lattice units)      */
  int periodic[3];               /* per axis; otherwise halfway bounce-back walls */
  double wall_velocity[6][3];    /* per face x-,x+,y-,y+,z-,z+ (moving walls)   */
  double fluid_body_force[3];    /* uniform Guo body force on the fluid (tests) */
  double gravity[3];             /* on particles, buoyancy-corrected            */
  int storage;                   /* MI_STORE_*                                  */
  int bb_mode;                   /* MI_BB_*                                     */
  int dem_substeps;              /* DEM substeps per LBM step, >= 1             */
  double kn, kt, eta_n, eta_t, mu_s; /* spring-dashpot contact parameters       */
  int guess_mode;                /* MI_GUESS_*                                  */
  int max_particles;             /* capacity of the particle table              */
  int max_balls;                 /* capacity of the metaball tables (all particles) */
  void *cuda_stream;             /* cudaStream_t to run on; NULL = a stream the handle creates */
  int device;                    /* CUDA device ordinal                         */
  /* Optional device allocator (e.g. a framework's caching allocator).  When
   * NULL, cudaMalloc / cudaFree are used.  dev_alloc returns NULL on failure. */
  void *(*dev_alloc)(size_t bytes, void *ctx);
  void (*dev_free)(void *ptr, size_t bytes, void *ctx);
  void *alloc_ctx;
  /* Nonzero: mi_delbm_add_particle rejects (MI_EOVERLAP) a particle whose
   * core overlaps an existing particle's, decided by the method's own closest-
   * point solve (Sec. 2.3.1): for every existing particle whose bounding
   * sphere meets the new one, plain Newton on grad(g_i + g_j) = 0 from the
   * plain guess, overlap when the converged point lies inside a core.
   * Default 0 (packed synthetic scenes and shape libraries add overlapping
   * particles on purpose). */
  int check_overlap;
} mi_delbm_config;

typedef struct mi_delbm mi_delbm;

/* ABI version of the loaded library (MI_DELBM_ABI_VERSION) and the size of
 * mi_delbm_config it was compiled with, so that bindings can check layout. */
int mi_delbm_abi_version(void);
size_t mi_delbm_config_size(void);

/* Fill *cfg with defaults: 64^3 closed box, tau 0.8, rho0 1, FP32 storage,
 * IBB, 1 DEM substep, kn 1, kt 2/7, eta_n = eta_t = 0, mu_s 0.4, plain guess,
 * 1024 particles, 65536 metaballs, device 0, handle-owned stream, cudaMalloc. */
void mi_delbm_config_init(mi_delbm_config *cfg);

/* Create a handle: allocates the two population buffers, node classes, owner
 * fields and lists on cfg->device, and sets every node to the rest state
 * f_i = w_i rho0 (post-collision populations at t = 0).
 * Errors: MI_EINVAL (bad sizes, tau <= 1/2, unknown modes), MI_ENOMEM, MI_ECUDA. */
mi_status mi_delbm_create(const mi_delbm_config *cfg, mi_delbm **out);

/* Free everything the handle owns (after synchronising its stream). NULL is a no-op. */
void mi_delbm_destroy(mi_delbm *h);

/* Message of the last failed call on this handle ("" if none).  Valid until
 * the next call on the handle.  h may be NULL (message of the last failed
 * mi_delbm_create on this thread). */
const char *mi_delbm_last_error(const mi_delbm *h);

/* Run n_steps full steps (all phases), asynchronously on the handle's stream.
 * Errors: MI_EINVAL (n_steps < 0), MI_ECUDA (launch failure). */
mi_status mi_delbm_step(mi_delbm *h, int n_steps);

/* Block the calling host thread until all work queued on the handle's stream
 * has finished; reports a pending device-side failure (MI_ECUDA). */
mi_status mi_delbm_synchronize(mi_delbm *h);

/* Run the listed phases of one step, in the fixed phase order, once.  Used by
 * tests to compare each phase with the oracle and by profilers.  A full step
 * is MI_PHASE_ALL.  Asynchronous. */
mi_status mi_delbm_step_phases(mi_delbm *h, unsigned phases);

/* Copy the current post-collision populations f_i (as float, [19][nz][ny][nx])
 * (the values at solid nodes are unspecified)
 * to or from the host.  For the deviation storages the stored value is
 * f_i - w_i rounded to the storage type on set, and w_i + stored on get (so a
 * get after a set returns the rounded value).  Synchronises.
 * count = 19*nx*ny*nz floats, else MI_EINVAL. */
mi_status mi_delbm_set_populations(mi_delbm *h, const float *host_f, size_t count);
mi_status mi_delbm_get_populations(mi_delbm *h, float *host_f, size_t count);

/* Raw stored populations (storage type, [19][nz][ny][nx], no conversion).
 * bytes = 19*nx*ny*nz*sizeof(storage element).  Synchronises. */
mi_status mi_delbm_set_raw_populations(mi_delbm *h, const void *host, size_t bytes);
mi_status mi_delbm_get_raw_populations(mi_delbm *h, void *host, size_t bytes);

/* Device addresses of the current state (for zero-copy inspection by a
 * framework; valid until the next call that steps or reallocates).
 * populations: element [q][z][y][x] at pop + q*plane_stride + ((z*ny + y)*nx + x),
 * in the storage type.  node_class: uint8 per node, bit 0 solid, bit 1
 * boundary (fluid with a solid neighbour), bit 2 newly uncovered.
 * owner: uint32 per node, particle index of a solid node, 0xFFFFFFFF if fluid. */
typedef struct {
  void *populations;
  size_t plane_stride;   /* elements between q planes */
  int storage;           /* MI_STORE_* */
  const uint8_t *node_class;
  const uint32_t *owner;
  void *stream;          /* cudaStream_t of the handle */
} mi_delbm_device_view;
mi_status mi_delbm_get_device_view(mi_delbm *h, mi_delbm_device_view *v);

/* ------------------------------------------------------------------------
 * Particles (Sec. 2.1 Eq. 1 shape; Sec. 2.3.1 rigid-body state)
 * ------------------------------------------------------------------------ */

/* Mass properties of a particle: mass, solid volume (buoyancy uses
 * rho0*volume) and inertia tensor in body axes about the body origin,
 * row-major. */
typedef struct {
  double mass;
  double volume;
  double inertia[9];
} mi_mass_props;

/* Add a rigid metaball particle: n_balls control points centers[n*3] (body
 * frame) with coefficients k[n] > 0 (the shape is f(x) = sum k_i/|x-c_i|^2 >= 1,
 * Eq. 1), density (fluid rho0 = 1 scale), sphero-metaball skin radius skin_Rs
 * (0 <= skin_Rs < sqrt(sum k)), pose pos[3] and unit quaternion quat[4]
 * (w, x, y, z; normalised by the library), velocity vel[3] and angular
 * velocity omega[3] (world frame).
 * mp == NULL: volume, centroid and inertia are integrated on the GPU by
 * midpoint quadrature of f >= 1 with spacing 1/4 lattice unit, the control
 * points are shifted so that the body origin is the centroid, and pos is
 * moved by R(quat) * centroid so that the particle does not move.
 * mp != NULL: the given mass properties are used and the body origin is taken
 * as the centroid (no shift).
 * On success *id_out is the particle index (0, 1, ... in order of addition).
 * Allowed between steps.  Errors: MI_EINVAL (bad values), MI_ECAPACITY
 * (max_particles / max_balls reached), MI_ENOMEM, MI_ECUDA. */
mi_status mi_delbm_add_particle(mi_delbm *h, int n_balls, const double *centers, const double *k,
                                double density, double skin_Rs, const double pos[3], const double quat[4],
                                const double vel[3], const double omega[3], const mi_mass_props *mp,
                                int *id_out);

/* Number of particles in the handle. */
int mi_delbm_num_particles(const mi_delbm *h);

/* Kinematic state of particle id (world frame).  get synchronises; set takes
 * effect at the next step (any pointer may be NULL to leave that part). */
mi_status mi_delbm_get_particle_state(mi_delbm *h, int id, double pos[3], double quat[4], double vel[3],
                                      double omega[3]);
mi_status mi_delbm_set_particle_state(mi_delbm *h, int id, const double pos[3], const double quat[4],
                                      const double vel[3], const double omega[3]);

/* Kinematic states of all particles as one array of n x 13 doubles per
 * particle [pos(3), quat(4), vel(3), omega(3)], copied asynchronously on the
 * handle's stream (use page-locked host memory for a true async copy).  n must
 * equal mi_delbm_num_particles.  set takes effect at the next step; get
 * returns the state after the work queued so far (synchronise before
 * reading the buffer). */
mi_status mi_delbm_set_particle_states(mi_delbm *h, const double *states, int n);
mi_status mi_delbm_get_particle_states(mi_delbm *h, double *states, int n);

/* Shape and mass properties of particle id as the library holds them (after
 * any centroid shift): centers[n*3], k[n] (cap entries available; *n_out is
 * the ball count), mass properties and bounding radius
 * R_b = max|c_i| + sqrt(sum k_i) (f < 1 beyond it).  Any output may be NULL. */
mi_status mi_delbm_get_particle_shape(mi_delbm *h, int id, double *centers, double *k, int cap, int *n_out,
                                      mi_mass_props *mp, double *Rb);

/* Hydrodynamic force and torque of the last step (momentum exchange, torque
 * about the particle position) and contact force and torque of the last DEM
 * substep, each num_particles x 3 doubles, caller-owned; any may be NULL.
 * Synchronises; reports MI_ECAPACITY if a list overflowed during the step. */
mi_status mi_delbm_forces(mi_delbm *h, double *F_hydro, double *T_hydro, double *F_contact, double *T_contact);

/* Contact candidates of the last DEM substep (Sec. 2.3.1): every broad-phase
 * pair i < j with |X_i - X_j| <= R_b,i + R_b,j + 1 and every particle-wall
 * item (j = -1 - face, faces x-,x+,y-,y+,z-,z+ at -1/2 and n - 1/2 of the
 * non-periodic axes) with its contact point xcp, unit normal n (pointing from
 * j to i, i.e. into particle i's side; the wall normal for walls), overlap
 * delta (> 0 means in contact and a force was applied), Newton iterations and
 * status (0 converged, 1 not converged, 2 singular Hessian, 3 closest point
 * inside a core, 4 out of range: no force in cases 1-4).  Order is
 * unspecified.  *n_out = number of candidates; MI_ECAPACITY (nothing written)
 * if it exceeds cap.  Synchronises. */
typedef struct {
  int i, j;
  double xcp[3], n[3], delta;
  int iters, status;
} mi_contact;
mi_status mi_delbm_contacts(mi_delbm *h, mi_contact *out, int cap, int *n_out);

/* Node classes (bit 0 solid, bit 1 boundary, bit 2 newly uncovered) and
 * owners (particle index of solid nodes, 0xFFFFFFFF for fluid) of the last
 * flag phase, count = nx*ny*nz entries each, [z][y][x]; either may be NULL.
 * Synchronises. */
mi_status mi_delbm_get_node_classes(mi_delbm *h, uint8_t *node_class, uint32_t *owner, size_t count);

/* Boundary links of the last flag phase: fluid node (linear index
 * (z*ny + y)*nx + x), direction d (1..18) towards the solid neighbour, its
 * particle, and the wall fraction q of the last links phase.  Order is
 * unspecified.  cap entries available per array; *n_out = number of links
 * (MI_ECAPACITY if larger than cap, nothing written).  Synchronises. */
mi_status mi_delbm_get_links(mi_delbm *h, size_t cap, int32_t *cell, int8_t *dir, int32_t *particle, float *q,
                             size_t *n_out);

/* Per-step counters of the last step (synchronises). status: bit 0..2 list
 * overflow (boundary nodes, links, uncovered nodes), bit 3 contact-pair
 * overflow, bit 4 contact overflow, bit 5 a particle moved more than two
 * nodes in one step; the bits are cleared by this call. */
typedef struct {
  long long boundary_nodes, links, new_nodes, candidate_pairs, contacts;
  unsigned status;
} mi_delbm_stats;
mi_status mi_delbm_get_stats(mi_delbm *h, mi_delbm_stats *st);

/* Set the capacities of the per-step lists exactly (boundary nodes, boundary
 * links, and uncovered nodes, which also bounds the covered-node list of the
 * cover/uncover rule), smaller or larger than the sizes mi_delbm_add_particle
 * estimates from the particles' boxes: for callers that budget device memory
 * (the lists take 12 B per boundary node, 13 B per link and 8 B per uncovered
 * node, plus 19 stored values per boundary node for the overlapped schedule).
 * A step whose lists overflow never writes past them: it completes with the
 * appends that fitted (its populations and forces are then incomplete), and
 * the next synchronising query (mi_delbm_forces, mi_delbm_contacts) returns
 * MI_ECAPACITY with the sizes it needed in the message; mi_delbm_get_stats
 * reports them as the counts.  Before the next step the handle grows the
 * lists to those sizes plus a quarter and captures its graphs again; restore
 * the state of the step that overflowed (populations, particle states) to
 * repeat it.  A later mi_delbm_add_particle may grow the lists again (never
 * shrinks them).  Synchronises.  Errors: MI_EINVAL (a capacity of 0 or above
 * 2^32 - 16), MI_ENOMEM. */
mi_status mi_delbm_reserve_lists(mi_delbm *h, size_t boundary_nodes, size_t links, size_t new_nodes);

/* State check: stored populations that are NaN or infinite at the nodes that
 * are not solid at the current flags (every node without particles; values
 * at solid nodes are unspecified), and particles whose position, quaternion,
 * velocity or angular velocity is not finite.  For 16-bit storages a value is
 * bad when its exponent bits are all ones.  Synchronises.  Returns MI_OK when
 * nothing is bad, MI_ESTATE (with the counts in the message and in *out)
 * otherwise.  first_bad_node is the linear index x + nx (y + ny z), -1 if
 * none. */
typedef struct {
  long long bad_populations, first_bad_node;
  int bad_particles, first_bad_particle;
} mi_delbm_health;
mi_status mi_delbm_check(mi_delbm *h, mi_delbm_health *out);

/* ------------------------------------------------------------------------
 * Allocation-free mass properties (the paper has no counterpart: this is a
 * library convenience for particular callers).
 *
 * mi_delbm_add_particle computes a particle's mass properties with scratch
 * memory it obtains from the handle's allocator.  Some callers cannot allow
 * that: code whose device memory is entirely reserved up front by another
 * allocator's pool (so a cudaMalloc would fail or fragment that pool), and
 * latency-critical loops that cannot afford the device-wide synchronisation
 * a cudaFree implies.  This entry point computes the same quantities -- the
 * same midpoint quadrature of f >= 1, with the same FP32 test and FP64 guard
 * band -- and allocates nothing: its scratch (an FP32 copy of at most 4096
 * balls and 1024 rows of 10 moment sums, about 144 KB) is a fixed static
 * array in device memory that every GPU which loads the library holds until
 * the process exits.
 *
 * balls_dev: device pointer, n_balls x 4 doubles (c_x, c_y, c_z, k) in the
 *   body frame, k > 0; 1 <= n_balls <= 4096 (MI_EINVAL otherwise: the static
 *   scratch holds no more).
 * density > 0; spacing > 0: the quadrature grid spacing (1/4 is what
 *   mi_delbm_add_particle uses).
 * out_dev: device pointer to 14 doubles, written as mass, volume,
 *   centroid[3], inertia[9] (row-major, about the centroid, body axes).
 *   All 14 are NaN when no sample lies inside the particle (no solid volume
 *   at this spacing), and when the grid is not run: the ball table is
 *   ill-formed (a NaN, a non-positive sum of k), or it has more than 2048
 *   samples per axis (ceil(2 R_b / spacing), R_b = max|c_i| + sqrt(sum k_i)),
 *   or more than 2^38 (sample, ball) pairs.  R_b is formed on the device, so
 *   these cases are reported through the outputs, not the return status.
 * stream: cudaStream_t to run on (NULL = the default stream).  The call is
 *   asynchronous; synchronise the stream before reading out_dev.
 * Runs on the current device.  The first call on a device looks up the
 *   scratch's device address (cudaGetSymbolAddress) once for that device and
 *   keeps it; make that first call before any stream capture.  The kept
 *   address belongs to the device's primary context of that time: after a
 *   cudaDeviceReset of the device, do not call this entry point on it again
 *   in the same process.
 * Every call on a device shares the one scratch array, which keeps the last
 *   call's contents: calls that overlap on the GPU (on different streams, or
 *   from different host threads) race and give wrong results.  Serialise them.
 * Errors (message via mi_delbm_last_error(NULL)): MI_EINVAL, MI_ECUDA.
 */
mi_status mi_mass_properties_noalloc(const double *balls_dev, int n_balls, double density, double spacing,
                                     double *out_dev, void *stream);

/* How mi_delbm_step runs its steps: 0 as individual launches; 1 (the
 * default) one CUDA graph launch per step: a graph of one whole step is
 * captured on first use for each parity of the alternating buffers and
 * replayed afterwards; 2 one graph launch for all the steps of a call: a
 * graph whose conditional while node repeats a body of two whole steps (both
 * parities) until a device counter, set before the launch, runs out; an odd
 * step count adds one single-step graph.  The three give the same bits.
 * Adding a particle, and every call documented to do so, discards the graphs.
 * While per-phase timing is enabled, steps run as individual launches.
 * Errors: MI_EINVAL (enable not 0, 1 or 2). */
mi_status mi_delbm_set_graphs(mi_delbm *h, int enable);

/* Choose the launch shapes of the bulk kernel (threads per block along x,
 * from 32/64/128/256) and of the list kernels (blocks per SM for the wall
 * fraction, refill and boundary-node kernels, from 2/4/8/16/32; the links'
 * bounce-back and the boundary nodes are timed together) by timing each candidate
 * with CUDA events on the handle's stream, and use the fastest from then on.
 * With cache_path != NULL, a line {"key": ..., "bulk_block_x": .., "list_blocks_per_sm": ..}
 * for this device, lattice, storage and particle count is read from that file
 * if present (no timing), else appended after timing.  The list kernels are
 * tuned only when the last step produced boundary nodes, so call this after
 * at least one step.  The trial launches leave the populations untouched and
 * clear the hydrodynamic force sums.  Synchronises; the chosen values are
 * returned through the non-NULL pointers. */
mi_status mi_delbm_autotune(mi_delbm *h, const char *cache_path, int *bulk_block_x, int *list_blocks_per_sm);

/* Step schedule flags. */
enum {
  /* the boundary nodes (interpolated bounce-back, momentum exchange,
   * collision) are computed on the particle side stream while the bulk kernel
   * runs, into a side buffer, and copied into the new populations after the
   * bulk and near kernels (the same bits as the default order, in which they
   * are computed after those kernels); steps that run all phases */
  MI_SCHEDULE_OVERLAP_BOUNDARY = 1,
  /* run the DEM substeps (dem_substeps > 1) as separate launches per
   * substep.  By default, with at most 64 particles and the plain or warm
   * start, one kernel runs all substeps of a step in one CTA (the same bits:
   * the same per-item and per-particle device code, no launch per substep) */
  MI_SCHEDULE_UNFUSED_DEM = 2,
  /* the links' interpolated bounce-back and momentum exchange run on the
   * particle side stream while the bulk kernel runs, instead of after it
   * (the same bits; the boundary nodes' collision still follows the bulk
   * kernel); steps that run the wall fractions, the refill and the boundary
   * phase.  Implied by MI_SCHEDULE_OVERLAP_BOUNDARY */
  MI_SCHEDULE_LINKS_BESIDE = 4
};
/* Set the step schedule (an OR of MI_SCHEDULE_* flags; 0 = default).
 * Discards captured graphs.  Errors: MI_EINVAL (unknown flags). */
mi_status mi_delbm_set_schedule(mi_delbm *h, int flags);

/* Momentum rule flags. */
enum {
  /* the covered/uncovered correction of Lorenz et al. (2009), whom Sec.
   * 2.3.2 cites with Chen (2013) for its momentum exchange: a node that a
   * particle covers this step (fluid before, solid now) hands the momentum
   * sum_i e_i f+_i(x, t) of its post-collision populations to that particle,
   * and a node that a particle uncovers takes the momentum of its refilled
   * populations from it; the forces and torques (arm x - X_p) join the
   * hydrodynamic sums that mi_delbm_forces returns.  The step that first
   * flags a particle (after mi_delbm_add_particle) covers nothing.  Off by
   * default (the paper describes no such term) */
  MI_MOMENTUM_COVER_UNCOVER = 1
};
/* Set the momentum rules (an OR of MI_MOMENTUM_* flags; 0 = default).
 * Discards captured graphs.  Errors: MI_EINVAL (unknown flags). */
mi_status mi_delbm_set_momentum_rules(mi_delbm *h, int flags);

/* Set the launch shapes directly (what mi_delbm_autotune chooses): bulk
 * kernel threads per block along x (32..256, a multiple of 32; at most 128
 * with pairs), rows per thread (1 or 2), paired nodes (0: no; 1 or 2: two
 * x-adjacent nodes per thread with paired accesses, used only when nx is
 * even; for 16-bit storages 1 and 2 select a 64- or 80-register budget;
 * 3: four x-adjacent nodes per thread with 64-bit accesses, 16-bit storages
 * with nx a multiple of 4 only, else the one-node kernel), list-kernel
 * blocks per SM (1..64).  Results do not depend on them. */
mi_status mi_delbm_set_tuning(mi_delbm *h, int bulk_block_x, int bulk_rows, int bulk_pairs, int list_blocks_per_sm);

/* The launch shapes in use (any pointer may be NULL). */
mi_status mi_delbm_get_tuning(const mi_delbm *h, int *bulk_block_x, int *bulk_rows, int *bulk_pairs,
                              int *list_blocks_per_sm);

/* Per-phase GPU timing with CUDA events on the handle's stream.  While
 * enabled, each launch of a phase inside mi_delbm_step is bracketed by events.
 * mi_delbm_phase_times synchronises and returns, per phase bit b (index b of
 * 8), the summed milliseconds and the number of timed launches since the last
 * reset (the reset flag clears them after reading). */
mi_status mi_delbm_set_timing(mi_delbm *h, int enable);
mi_status mi_delbm_phase_times(mi_delbm *h, double ms[8], long long launches[8], int reset);
/* The same event timing for one kernel: the summed milliseconds and count of
 * the timed launches of `kernel` since the last reset of mi_delbm_phase_times
 * (not reset by this call).  Names: k_prologue, k_clear, k_flag, k_classify,
 * k_links_q, k_refill, k_bulk (the bulk stream-collide, whichever variant the
 * tuning selects), k_near, k_links_ibb, k_boundary, k_scatter_boundary, k_dem_prologue,
 * k_broad_phase, k_item_features, k_mlp_tc, k_contacts, k_integrate,
 * k_dem_substeps.  Synchronises.  Errors: MI_EINVAL (NULL argument). */
mi_status mi_delbm_kernel_time(mi_delbm *h, const char *kernel, double *ms, long long *launches);

/* Number of kernel launches the handle issued since creation (for launch
 * accounting by benchmarks). */
long long mi_delbm_launch_count(const mi_delbm *h);

/* ------------------------------------------------------------------------
 * Learned Newton guess.  Not in the paper: its closest-point solve (Sec.
 * 2.3.1, Newton-Raphson on grad(g_i + g_j) = 0 between the two cores) starts
 * from a heuristic point.  Here a small network, trained on solves the
 * method itself makes, proposes the starting point and the balls that matter
 * near the solution; full-set Newton to the unchanged tolerance still decides
 * the result, and plain Newton from the plain guess takes over whenever the
 * learned start does not converge.
 *
 * Network: 64 -> 256 -> 256 -> 4, ReLU after both hidden layers.  Parameters
 * are one FP32 array of mi_mlp_param_count() floats: W1 (64 x 256, row-major,
 * input index first), b1 (256), W2 (256 x 256), b2 (256), W3 (256 x 4), b3 (4).
 * Every product runs on the tensor cores with BF16 operands and FP32
 * accumulation; activations, gradients and the AdamW state stay FP32.
 *
 * Features of a pair (64, lengths over L = max(R_b,i, R_b,j), positions
 * relative to O = (X_i + X_j)/2): 0:3 (X_j - X_i)/L; 3:7, 7:11 unit
 * quaternions with w >= 0; 11:14 (x_a - O)/L with x_a the anchor (midpoint of
 * the surface points of the ball of i whose sphere, radius sqrt k, reaches
 * closest to X_j and the ball of j reaching closest to X_i); 14:16 log g_i,
 * log g_j at x_a; 16:40 and 40:64 per particle log(n)/5, log(sum k / L^2),
 * R_b/L, R_s/L and, for the 5 balls nearest x_a (ties to the lower index,
 * zeros when fewer), (c - x_a)/L and log(s k / L^2), s the core scale.
 * Outputs: (x_m - x_a)/L and log(r_act/L).  The start is x_a + L (out 0:3);
 * Newton first runs on the balls within L exp(out 3) of it.
 * ---------------------------------------------------------------------- */

/* Floats in the parameter array (83,460). */
size_t mi_mlp_param_count(void);

/* Y (n x 4) = MLP(X (n x 64)); acts (n x 512 floats, device) receives the two
 * hidden layers after ReLU for mi_mlp_backward.  All pointers are device
 * pointers; asynchronous on stream (a cudaStream_t, NULL: the legacy default
 * stream).  n == 0 does nothing (the pointers may then be NULL).  Errors:
 * MI_EINVAL (null pointer, n < 0), MI_ECUDA (launch). */
mi_status mi_mlp_forward(const float *params, const float *X, int n, float *Y, float *acts, void *stream);

/* Loss = (1/n) sum over rows and outputs of (Y - T)^2 into *loss (device),
 * and dY = dLoss/dY (n x 4).  scratch: 64 doubles of device memory. */
mi_status mi_mlp_mse(const float *Y, const float *T, int n, float *dY, float *loss, double *scratch, void *stream);

/* Gradients of the loss with respect to every parameter (same layout as the
 * parameters) from X, the acts of mi_mlp_forward and dY.  scratch: n x 512
 * floats of device memory.  Deterministic (no atomics). */
mi_status mi_mlp_backward(const float *params, const float *X, const float *acts, const float *dY, int n,
                          float *grads, float *scratch, void *stream);

/* One AdamW step (decoupled weight decay) over all parameters; m and v are
 * the moment arrays (zero before the first step), step the 1-based count. */
mi_status mi_mlp_adamw(float *params, const float *grads, float *m, float *v, int step, float lr, float beta1,
                       float beta2, float eps, float weight_decay, void *stream);

/* Column-wise affine map of a row-major n x cols device array, in place:
 * X[r][c] = (X[r][c] - shift[c]) * scale[c] (shift, scale: cols device
 * floats).  The training driver standardises the features and weights the
 * targets with it.  Asynchronous on stream.  Errors: MI_EINVAL, MI_ECUDA. */
mi_status mi_mlp_scale_columns(float *X, long long n, int cols, const float *shift, const float *scale, void *stream);

/* Fused inference: the parameters packed once into a BF16 image of
 * mi_mlp_image_bytes() bytes (device, 16-byte aligned, owned by the caller),
 * then Y (n x 4) = MLP(X (n x 64)) by one persistent kernel.
 * mi_mlp_infer (the path the contact phase takes) runs on the tcgen05 tensor
 * cores: 128-row tiles, the FP32 accumulator in tensor memory, the weights
 * streamed through shared memory by bulk copies; if one of its bounded waits
 * gives up, the rows it did not finish are written as NaN.  mi_mlp_infer_mma
 * runs the same network with mma.sync, the whole network resident in shared
 * memory.  Both use the same BF16 operands as mi_mlp_forward; the FP32 sums
 * run in other orders, so the three agree to FP32 rounding.  X and Y 16-byte
 * aligned; n == 0 does nothing.  Errors: MI_EINVAL (null or misaligned
 * pointer, n < 0), MI_ECUDA. */
size_t mi_mlp_image_bytes(void);
mi_status mi_mlp_pack(const float *params, void *image, void *stream);
mi_status mi_mlp_infer(const void *image, const float *X, int n, float *Y, void *stream);
mi_status mi_mlp_infer_mma(const void *image, const float *X, int n, float *Y, void *stream);

/* Contact guess of the handle's DEM substeps: MI_GUESS_PLAIN, MI_GUESS_WARM
 * (params ignored), or MI_GUESS_LEARNED with params (device,
 * mi_mlp_param_count floats, packed into the handle; the caller keeps
 * ownership of its array).  Wall contacts always
 * start from the plain guess.  Discards captured graphs.  Errors: MI_EINVAL,
 * MI_ENOMEM, MI_ECUDA. */
mi_status mi_delbm_set_guess(mi_delbm *h, int mode, const float *params);

/* Bounded waits of the learned guess's tcgen05 inference kernel: every wait on
 * its copies and tensor-core work gives up after wait_rounds mbarrier polls
 * (0: the default, 2^24, well over a second); a wait that gives up marks the
 * rows it did not finish NaN, the contacts of those rows fall back to plain
 * Newton from the plain guess, and the next synchronising query returns
 * MI_ETIMEOUT (mi_delbm_get_stats clears it).  stall != 0 is for
 * fault-injection tests: before issuing any work the kernel waits on an
 * mbarrier that nothing arrives at, so that this wait runs out (after
 * wait_rounds polls) with no copy or MMA in flight.  Discards the captured
 * graphs. */
mi_status mi_delbm_set_guess_wait(mi_delbm *h, unsigned wait_rounds, int stall);

/* Flags of mi_delbm_pair_solve. */
enum {
  MI_PAIR_FEATURES = 1,  /* write the 64 features of each pair into X          */
  MI_PAIR_PLAIN = 2,     /* solve from the plain guess                          */
  MI_PAIR_LEARNED = 4,   /* solve from the learned start (pred; X holds the
                            features, computed now when MI_PAIR_FEATURES is set) */
  MI_PAIR_LABELS = 8,    /* write the training targets of converged pairs to T  */
  MI_PAIR_GUESS_ONLY = 16 /* with PLAIN: stop at the plain guess (Sec. 2.3.1's
                            starting point): xm = that point, iters = evals = 0,
                            status 0; no LABELS                                 */
};

/* Closest points of n explicitly posed pairs of the handle's particle shapes,
 * one warp per pair, asynchronously on the handle's stream; the lattice and
 * the particles' own states are not touched.  Device arrays: ij (n x 2
 * particle indices, which give the shapes), poses (n x 14 doubles: pos_i,
 * quat_i, pos_j, quat_j), pred (n x 4, LEARNED), X (n x 64, FEATURES or
 * LEARNED), T (n x 4, LABELS; rows of unconverged pairs untouched), and the
 * outputs xm (n x 3 doubles, world closest point x_m), iters (Newton
 * iterations, subset + full set + fallback), evals (ball evaluations of those
 * iterations), status (0 converged, 1 not converged, 2 singular, 3 inside a
 * core, 4 out of range, 5 bad index; +16 when the learned start fell back to
 * plain Newton).  xm, iters, evals and status may be NULL only when neither
 * PLAIN nor LEARNED is set.  Errors: MI_EINVAL (flags, null pointers),
 * MI_ECUDA. */
mi_status mi_delbm_pair_solve(mi_delbm *h, int n, const int *ij, const double *poses, int flags, const float *pred,
                              float *X, float *T, double *xm, int *iters, int *evals, int *status);

#ifdef __cplusplus
}
#endif

#endif /* MI_DELBM_H */
