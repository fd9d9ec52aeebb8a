"""ctypes binding of libmi_delbm (the C-ABI declared in include/mi_delbm.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch, when used, only provides device memory (its caching
allocator is plugged into the handle through the config's dev_alloc/dev_free
callbacks) and the CUDA stream.  There is no CPU fallback: if the shared
library is missing this module raises ImportError.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmi_delbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libmi_delbm.so is not built (expected at %s); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` first" % LIB_PATH)

lib = ctypes.CDLL(LIB_PATH)

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p)

MI_OK, MI_EINVAL, MI_ENOMEM, MI_ECUDA, MI_ECAPACITY, MI_EOVERLAP, MI_ESTATE, MI_ETIMEOUT, MI_ENOTSUP = range(9)
STATUS_NAMES = ["MI_OK", "MI_EINVAL", "MI_ENOMEM", "MI_ECUDA", "MI_ECAPACITY", "MI_EOVERLAP",
                "MI_ESTATE", "MI_ETIMEOUT", "MI_ENOTSUP"]
STORE_F32, STORE_F16_DEV, STORE_BF16_DEV = 0, 1, 2
BB_IBB, BB_LADD = 0, 1
GUESS_PLAIN, GUESS_LEARNED, GUESS_WARM = 0, 1, 2
PHASE_FLAG, PHASE_LINKS, PHASE_REFILL, PHASE_BULK = 1, 2, 4, 8
PHASE_BOUNDARY, PHASE_SWAP, PHASE_CONTACT, PHASE_INTEGRATE = 16, 32, 64, 128
PHASE_ALL = 0xFF
PHASE_NAMES = ["flag", "links", "refill", "bulk", "boundary", "swap", "contact", "integrate"]


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("nz", c_int),
        ("tau", c_double), ("rho0", c_double),
        ("periodic", c_int * 3),
        ("wall_velocity", (c_double * 3) * 6),
        ("fluid_body_force", c_double * 3),
        ("gravity", c_double * 3),
        ("storage", c_int), ("bb_mode", c_int), ("dem_substeps", c_int),
        ("kn", c_double), ("kt", c_double), ("eta_n", c_double), ("eta_t", c_double), ("mu_s", c_double),
        ("guess_mode", c_int), ("max_particles", c_int), ("max_balls", c_int),
        ("cuda_stream", c_void_p), ("device", c_int),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", c_void_p),
        ("check_overlap", c_int),
    ]


class Health(ctypes.Structure):
    _fields_ = [("bad_populations", ctypes.c_longlong), ("first_bad_node", ctypes.c_longlong),
                ("bad_particles", c_int), ("first_bad_particle", c_int)]


class DeviceView(ctypes.Structure):
    _fields_ = [("populations", c_void_p), ("plane_stride", c_size_t), ("storage", c_int),
                ("node_class", c_void_p), ("owner", c_void_p), ("stream", c_void_p)]


class MassProps(ctypes.Structure):
    _fields_ = [("mass", c_double), ("volume", c_double), ("inertia", c_double * 9)]


class Stats(ctypes.Structure):
    _fields_ = [("boundary_nodes", ctypes.c_longlong), ("links", ctypes.c_longlong),
                ("new_nodes", ctypes.c_longlong), ("candidate_pairs", ctypes.c_longlong),
                ("contacts", ctypes.c_longlong), ("status", ctypes.c_uint)]


class Contact(ctypes.Structure):
    _fields_ = [("i", c_int), ("j", c_int), ("xcp", c_double * 3), ("n", c_double * 3), ("delta", c_double),
                ("iters", c_int), ("status", c_int)]


def _sig(name, restype, *argtypes):
    fn = getattr(lib, name)
    fn.restype = restype
    fn.argtypes = list(argtypes)
    return fn


_P = c_void_p
_sig("mi_delbm_abi_version", c_int)
_sig("mi_delbm_config_size", c_size_t)
_sig("mi_delbm_config_init", None, ctypes.POINTER(Config))
_sig("mi_delbm_create", c_int, ctypes.POINTER(Config), ctypes.POINTER(c_void_p))
_sig("mi_delbm_destroy", None, _P)
_sig("mi_delbm_last_error", ctypes.c_char_p, _P)
_sig("mi_delbm_step", c_int, _P, c_int)
_sig("mi_delbm_step_phases", c_int, _P, ctypes.c_uint)
_sig("mi_delbm_synchronize", c_int, _P)
_sig("mi_delbm_set_populations", c_int, _P, _P, c_size_t)
_sig("mi_delbm_get_populations", c_int, _P, _P, c_size_t)
_sig("mi_delbm_set_raw_populations", c_int, _P, _P, c_size_t)
_sig("mi_delbm_get_raw_populations", c_int, _P, _P, c_size_t)
_sig("mi_delbm_get_device_view", c_int, _P, ctypes.POINTER(DeviceView))
_sig("mi_delbm_set_timing", c_int, _P, c_int)
_sig("mi_delbm_set_graphs", c_int, _P, c_int)
_sig("mi_delbm_set_tuning", c_int, _P, c_int, c_int, c_int, c_int)
_sig("mi_delbm_get_tuning", c_int, _P, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
     ctypes.POINTER(c_int))
_sig("mi_delbm_autotune", c_int, _P, ctypes.c_char_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int))
_sig("mi_delbm_phase_times", c_int, _P, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong), c_int)
_sig("mi_delbm_reserve_lists", c_int, _P, c_size_t, c_size_t, c_size_t)
_sig("mi_delbm_set_guess_wait", c_int, _P, ctypes.c_uint, c_int)
_sig("mi_delbm_check", c_int, _P, _P)
_sig("mi_delbm_kernel_time", c_int, _P, ctypes.c_char_p, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong))
_sig("mi_delbm_launch_count", ctypes.c_longlong, _P)
_sig("mi_delbm_add_particle", c_int, _P, c_int, _P, _P, c_double, c_double, _P, _P, _P, _P,
     ctypes.POINTER(MassProps), ctypes.POINTER(c_int))
_sig("mi_delbm_num_particles", c_int, _P)
_sig("mi_delbm_get_particle_state", c_int, _P, c_int, _P, _P, _P, _P)
_sig("mi_delbm_set_particle_state", c_int, _P, c_int, _P, _P, _P, _P)
_sig("mi_delbm_set_particle_states", c_int, _P, _P, c_int)
_sig("mi_delbm_get_particle_states", c_int, _P, _P, c_int)
_sig("mi_delbm_get_particle_shape", c_int, _P, c_int, _P, _P, c_int, ctypes.POINTER(c_int),
     ctypes.POINTER(MassProps), ctypes.POINTER(c_double))
_sig("mi_delbm_forces", c_int, _P, _P, _P, _P, _P)
_sig("mi_delbm_get_node_classes", c_int, _P, _P, _P, c_size_t)
_sig("mi_delbm_get_links", c_int, _P, c_size_t, _P, _P, _P, _P, ctypes.POINTER(c_size_t))
_sig("mi_delbm_get_stats", c_int, _P, ctypes.POINTER(Stats))
_sig("mi_delbm_contacts", c_int, _P, ctypes.POINTER(Contact), c_int, ctypes.POINTER(c_int))
_sig("mi_mass_properties_noalloc", c_int, _P, c_int, c_double, c_double, _P, _P)
_sig("mi_measure_fma_peak", c_int, c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_double), _P)
_sig("mi_mlp_param_count", c_size_t)
_sig("mi_mlp_forward", c_int, _P, _P, c_int, _P, _P, _P)
_sig("mi_mlp_mse", c_int, _P, _P, c_int, _P, _P, _P, _P)
_sig("mi_mlp_backward", c_int, _P, _P, _P, _P, c_int, _P, _P, _P)
_sig("mi_mlp_scale_columns", c_int, _P, ctypes.c_longlong, c_int, _P, _P, _P)
_sig("mi_mlp_adamw", c_int, _P, _P, _P, _P, c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
     ctypes.c_float, _P)
_sig("mi_mlp_image_bytes", c_size_t)
_sig("mi_mlp_pack", c_int, _P, _P, _P)
_sig("mi_mlp_infer", c_int, _P, _P, c_int, _P, _P)
_sig("mi_mlp_infer_mma", c_int, _P, _P, c_int, _P, _P)
_sig("mi_delbm_set_guess", c_int, _P, c_int, _P)
_sig("mi_delbm_set_schedule", c_int, _P, c_int)
_sig("mi_delbm_set_momentum_rules", c_int, _P, c_int)
_sig("mi_shape_scratch_bytes", ctypes.c_size_t, c_int, c_int)
_sig("mi_shape_descriptors", c_int, c_int, _P, _P, _P, _P, c_int, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P)
_sig("mi_ga_scratch_bytes", ctypes.c_size_t, c_int, c_int)
_sig("mi_ga_run", c_int, c_int, c_int, _P, c_int, _P, c_int, _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_ulonglong, c_int, c_int, _P, _P, _P, _P, _P, _P)
_sig("mi_gs_fit", c_int, c_int, _P, _P, _P, _P, _P, _P, c_int, c_int, c_int, ctypes.c_float, _P, _P, _P)
_sig("mi_delbm_pair_solve", c_int, _P, c_int, _P, _P, c_int, _P, _P, _P, _P, _P, _P, _P)

PAIR_FEATURES, PAIR_PLAIN, PAIR_LEARNED, PAIR_LABELS, PAIR_GUESS_ONLY = 1, 2, 4, 8, 16
SCHEDULE_OVERLAP_BOUNDARY, SCHEDULE_UNFUSED_DEM, SCHEDULE_LINKS_BESIDE = 1, 2, 4
MOMENTUM_COVER_UNCOVER = 1


def measure_fma_peak(precision="fp32", stream=None):
    """Measured dense FMA throughput of the current device (mi_measure_fma_peak):
    (TFLOP/s, ms of the timed launch)."""
    tf, ms = c_double(0.0), c_double(0.0)
    st = lib.mi_measure_fma_peak({"fp32": 0, "fp64": 1}[precision], ctypes.byref(tf), ctypes.byref(ms),
                                 c_void_p(int(stream) if stream else 0))
    if st != MI_OK:
        raise MiDelbmError(st, lib.mi_delbm_last_error(None).decode())
    return tf.value, ms.value


def mass_properties_noalloc(balls_dev_ptr, n_balls, density, spacing, out_dev_ptr, stream=None):
    """Allocation-free mass properties: device input n x 4 doubles, device
    output 14 doubles (mass, volume, centroid[3], inertia[9]); asynchronous
    on `stream` (a cudaStream_t handle as int, or None)."""
    st = lib.mi_mass_properties_noalloc(c_void_p(int(balls_dev_ptr)), int(n_balls), float(density), float(spacing),
                                        c_void_p(int(out_dev_ptr)), c_void_p(int(stream)) if stream else None)
    if st != MI_OK:
        raise MiDelbmError(st, lib.mi_delbm_last_error(None).decode())

def _tp(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    return c_void_p(t.data_ptr()) if t is not None else None


def _cur_stream():
    import torch
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _mlp_check(st):
    if st != MI_OK:
        raise MiDelbmError(st, lib.mi_delbm_last_error(None).decode())


def mlp_param_count():
    return int(lib.mi_mlp_param_count())


def mlp_forward(params, X):
    """Y (n x 4) and the saved activations (n x 512) for X (n x 64), all
    float32 CUDA tensors, on torch's current stream."""
    import torch
    n = X.shape[0]
    Y = torch.empty((n, 4), dtype=torch.float32, device=X.device)
    acts = torch.empty((n, 512), dtype=torch.float32, device=X.device)
    _mlp_check(lib.mi_mlp_forward(_tp(params), _tp(X), int(n), _tp(Y), _tp(acts), _cur_stream()))
    return Y, acts


def mlp_pack(params):
    """The packed BF16 image of the parameters for mlp_infer (uint8 CUDA tensor)."""
    import torch
    img = torch.empty(int(lib.mi_mlp_image_bytes()), dtype=torch.uint8, device=params.device)
    _mlp_check(lib.mi_mlp_pack(_tp(params), _tp(img), _cur_stream()))
    return img


def mlp_infer(image, X, engine="tcgen05"):
    """Y (n x 4) for X (n x 64) through the fused inference kernel
    (engine "tcgen05" or "mma")."""
    import torch
    n = X.shape[0]
    Y = torch.empty((n, 4), dtype=torch.float32, device=X.device)
    fn = lib.mi_mlp_infer if engine == "tcgen05" else lib.mi_mlp_infer_mma
    _mlp_check(fn(_tp(image), _tp(X), int(n), _tp(Y), _cur_stream()))
    return Y


GS_MAX_POINTS, GS_MAX_BALLS = 10240, 256


def gs_fit(hulls, models, planes, epochs, lr):
    """Gradient Search refinement (mi_gs_fit) of several models at once.
    hulls: list of (m_f, 3) point arrays, models: list of (c (n_f, 3), k
    (n_f,)), planes: list of (p_f, 4) facet planes; host arrays, copied to the
    device in one batch.  Returns a list of (c, k, active) per fit and the
    (n_fits, 2) losses after the first and the second descent."""
    import torch
    nf = len(hulls)
    dev = torch.device("cuda")

    def cat(arrs, width):
        a = np.concatenate([np.asarray(x, dtype=np.float32).reshape(-1, width) for x in arrs])
        off = np.concatenate([[0], np.cumsum([len(np.asarray(x).reshape(-1, width)) for x in arrs])]).astype(np.int32)
        return torch.as_tensor(a, device=dev).contiguous(), torch.as_tensor(off, device=dev)

    H, hoff = cat(hulls, 3)
    M, boff = cat([np.concatenate([np.asarray(c, np.float32).reshape(-1, 3), np.asarray(k, np.float32).reshape(-1, 1)],
                                  1) for c, k in models], 4)
    P, poff = cat(planes, 4)
    active = torch.empty(M.shape[0], dtype=torch.int32, device=dev)
    loss = torch.empty((nf, 2), dtype=torch.float32, device=dev)
    mp = max(len(np.asarray(h).reshape(-1, 3)) for h in hulls)
    mb = max(len(np.asarray(k).reshape(-1)) for _, k in models)
    _mlp_check(lib.mi_gs_fit(nf, _tp(hoff), _tp(H), _tp(boff), _tp(M), _tp(poff), _tp(P), int(mp), int(mb),
                             int(epochs), float(lr), _tp(active), _tp(loss), _cur_stream()))
    torch.cuda.synchronize()
    Mh, ah, bo = M.cpu().numpy(), active.cpu().numpy(), boff.cpu().numpy()
    out = [(Mh[bo[f]:bo[f + 1], :3], Mh[bo[f]:bo[f + 1], 3], ah[bo[f]:bo[f + 1]].astype(bool)) for f in range(nf)]
    return out, loss.cpu().numpy()


def ga_run(hull, planes, bbox, krange, n_ind, n_genes, generations, c_m, c_c, seed, pop=None):
    """Genetic Algorithm capture (mi_ga_run) on one hull: host arrays in,
    host arrays out: (population (n_ind, n_genes, 4), fitness (n_ind,),
    children of the last generation, their fitness).  pop=None draws the
    initial population on the device."""
    import torch
    dev = torch.device("cuda")
    H = torch.as_tensor(np.asarray(hull, dtype=np.float32).reshape(-1, 3), device=dev).contiguous()
    P = torch.as_tensor(np.asarray(planes, dtype=np.float32).reshape(-1, 4), device=dev).contiguous()
    if pop is None:
        Pop = torch.empty((n_ind, n_genes, 4), dtype=torch.float32, device=dev)
    else:
        Pop = torch.as_tensor(np.asarray(pop, dtype=np.float32).reshape(n_ind, n_genes, 4), device=dev).contiguous()
    fit = torch.empty(n_ind, dtype=torch.float32, device=dev)
    off = torch.empty_like(Pop)
    fo = torch.empty(n_ind, dtype=torch.float32, device=dev)
    scratch = torch.empty(int(lib.mi_ga_scratch_bytes(n_ind, n_genes)), dtype=torch.uint8, device=dev)
    bb = (ctypes.c_float * 6)(*[float(v) for v in np.asarray(bbox, dtype=np.float32)])
    kr = (ctypes.c_float * 2)(*[float(v) for v in np.asarray(krange, dtype=np.float32)])
    _mlp_check(lib.mi_ga_run(int(n_ind), int(n_genes), _tp(H), int(H.shape[0]), _tp(P), int(P.shape[0]), ctypes.cast(bb, c_void_p), ctypes.cast(kr, c_void_p),
                             float(c_m), float(c_c), int(seed), int(generations), 1 if pop is None else 0, _tp(Pop),
                             _tp(fit), _tp(off), _tp(fo), _tp(scratch), _cur_stream()))
    torch.cuda.synchronize()
    return Pop.cpu().numpy(), fit.cpu().numpy(), off.cpu().numpy(), fo.cpu().numpy()


SHAPE_FIELDS = ("volume", "surface", "l_long", "l_int", "l_short", "projected_area", "sphericity", "d_n", "d_s",
                "csf", "cells")


def shape_descriptors(models, h, eps=0.1):
    """Shape descriptors (mi_shape_descriptors) of metaball models given as
    (centres (n, 3), k (n,)) in their body frames: a list of dicts with
    SHAPE_FIELDS and the principal axes (rows, longest first).  The grid of
    each model spans +-R_g, R_g = max |c| + sqrt(sum k / (1 - eps)), rounded
    to FP32, with ceil(2 R_g / h) cells per axis."""
    import torch
    dev = torch.device("cuda")
    rg, ng, rows = [], [], []
    for c, k in models:
        c = np.asarray(c, dtype=np.float32).reshape(-1, 3)
        k = np.asarray(k, dtype=np.float32).reshape(-1)
        c64, k64 = c.astype(np.float64), k.astype(np.float64)
        r = np.float32(float(np.sqrt((c64 * c64).sum(1)).max() + np.sqrt(k64.sum() / (1.0 - eps))))
        rg.append(r)
        ng.append(int(np.ceil(2.0 * float(r) / h)))
        rows.append(np.concatenate([c, k[:, None]], 1))
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    balls = torch.as_tensor(np.concatenate(rows), device=dev).contiguous()
    offs = torch.as_tensor(off, device=dev)
    R = torch.as_tensor(np.array(rg, dtype=np.float32), device=dev)
    N = torch.as_tensor(np.array(ng, dtype=np.int32), device=dev)
    npart, max_n = len(models), max(ng)
    out = torch.empty((npart, len(SHAPE_FIELDS)), dtype=torch.float64, device=dev)
    axes = torch.empty((npart, 9), dtype=torch.float32, device=dev)
    scratch = torch.empty(int(lib.mi_shape_scratch_bytes(npart, max_n)), dtype=torch.uint8, device=dev)
    _mlp_check(lib.mi_shape_descriptors(npart, _tp(offs), _tp(balls), _tp(R), _tp(N), int(max_n), float(h),
                                        float(eps), _tp(out), _tp(axes), _tp(scratch), _cur_stream()))
    torch.cuda.synchronize()
    o, a = out.cpu().numpy(), axes.cpu().numpy()
    res = []
    for p in range(npart):
        d = {f: float(o[p, i]) for i, f in enumerate(SHAPE_FIELDS)}
        d["axes"] = a[p].reshape(3, 3)
        res.append(d)
    return res


def mlp_mse(Y, T):
    """(loss as a 1-element device tensor, dY)."""
    import torch
    n = Y.shape[0]
    dY = torch.empty_like(Y)
    loss = torch.empty(1, dtype=torch.float32, device=Y.device)
    scratch = torch.empty(64, dtype=torch.float64, device=Y.device)
    _mlp_check(lib.mi_mlp_mse(_tp(Y), _tp(T), int(n), _tp(dY), _tp(loss), _tp(scratch), _cur_stream()))
    return loss, dY


def mlp_backward(params, X, acts, dY):
    """Gradients (same layout as params)."""
    import torch
    n = X.shape[0]
    grads = torch.empty_like(params)
    scratch = torch.empty((n, 512), dtype=torch.float32, device=X.device)
    _mlp_check(lib.mi_mlp_backward(_tp(params), _tp(X), _tp(acts), _tp(dY), int(n), _tp(grads), _tp(scratch),
                                   _cur_stream()))
    return grads


def mlp_scale_columns(X, shift, scale):
    """In place X[r][c] = (X[r][c] - shift[c]) * scale[c] on a row-major CUDA
    float32 tensor; shift and scale are float32 CUDA tensors of X.shape[1]."""
    _mlp_check(lib.mi_mlp_scale_columns(_tp(X), int(X.shape[0]), int(X.shape[1]), _tp(shift), _tp(scale),
                                        _cur_stream()))


def mlp_adamw(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
    """One in-place AdamW step of params (m, v: moment tensors)."""
    _mlp_check(lib.mi_mlp_adamw(_tp(params), _tp(grads), _tp(m), _tp(v), int(step), float(lr), float(beta1),
                                float(beta2), float(eps), float(weight_decay), _cur_stream()))


if lib.mi_delbm_abi_version() != 2:
    raise ImportError("libmi_delbm ABI version mismatch")
if lib.mi_delbm_config_size() != ctypes.sizeof(Config):
    raise ImportError("mi_delbm_config layout mismatch: C %d bytes, binding %d bytes"
                      % (lib.mi_delbm_config_size(), ctypes.sizeof(Config)))


class MiDelbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


def _ptr(a):
    return a.ctypes.data_as(c_void_p)


class _TorchAllocator:
    """Routes the handle's device allocations to torch's caching allocator."""

    def __init__(self, device, stream):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None

    def _free(self, ptr, nbytes, ctx):
        try:
            self._torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


class Simulation:
    """One lattice and its particles on one GPU (a mi_delbm handle)."""

    def __init__(self, nx=64, ny=64, nz=64, tau=0.8, rho0=1.0, periodic=(False, False, False),
                 wall_velocity=None, fluid_body_force=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0),
                 storage=STORE_F32, bb_mode=BB_IBB, dem_substeps=1, kn=1.0, kt=2.0 / 7.0,
                 eta_n=0.0, eta_t=0.0, mu_s=0.4, guess_mode=GUESS_PLAIN, max_particles=1024,
                 max_balls=65536, device=0, stream=None, torch_memory=True, check_overlap=False):
        cfg = Config()
        lib.mi_delbm_config_init(ctypes.byref(cfg))
        cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
        cfg.tau, cfg.rho0 = float(tau), float(rho0)
        for a in range(3):
            cfg.periodic[a] = 1 if periodic[a] else 0
            cfg.fluid_body_force[a] = float(fluid_body_force[a])
            cfg.gravity[a] = float(gravity[a])
        if wall_velocity is not None:
            wv = np.asarray(wall_velocity, dtype=np.float64).reshape(6, 3)
            for f in range(6):
                for a in range(3):
                    cfg.wall_velocity[f][a] = wv[f, a]
        cfg.storage, cfg.bb_mode, cfg.dem_substeps = int(storage), int(bb_mode), int(dem_substeps)
        cfg.kn, cfg.kt, cfg.eta_n, cfg.eta_t, cfg.mu_s = float(kn), float(kt), float(eta_n), float(eta_t), float(mu_s)
        cfg.guess_mode, cfg.max_particles, cfg.max_balls = int(guess_mode), int(max_particles), int(max_balls)
        cfg.device = int(device)
        cfg.check_overlap = 1 if check_overlap else 0
        self._alloc = None
        self.torch_stream = None
        if stream is None and torch_memory:
            import torch
            self.torch_stream = torch.cuda.Stream(device=device)
            stream = self.torch_stream.cuda_stream
        if stream is not None:
            cfg.cuda_stream = c_void_p(int(stream))
        if torch_memory:
            self._alloc = _TorchAllocator(int(device), int(stream) if stream is not None else 0)
            cfg.dev_alloc = self._alloc.alloc
            cfg.dev_free = self._alloc.free
        self.cfg = cfg
        self.shape = (int(nz), int(ny), int(nx))
        self.ncell = int(nx) * int(ny) * int(nz)
        h = c_void_p()
        st = lib.mi_delbm_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != MI_OK:
            raise MiDelbmError(st, lib.mi_delbm_last_error(None).decode())
        self.h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.mi_delbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != MI_OK:
            raise MiDelbmError(st, lib.mi_delbm_last_error(self.h).decode())

    # -- stepping ---------------------------------------------------------
    def step(self, n=1):
        self._check(lib.mi_delbm_step(self.h, int(n)))

    def synchronize(self):
        self._check(lib.mi_delbm_synchronize(self.h))

    def step_phases(self, phases):
        self._check(lib.mi_delbm_step_phases(self.h, int(phases)))

    # -- populations ------------------------------------------------------
    def set_populations(self, f):
        a = np.ascontiguousarray(f, dtype=np.float32).reshape(19, *self.shape)
        self._check(lib.mi_delbm_set_populations(self.h, _ptr(a), a.size))

    def get_populations(self):
        a = np.empty((19,) + self.shape, dtype=np.float32)
        self._check(lib.mi_delbm_get_populations(self.h, _ptr(a), a.size))
        return a

    def set_raw_populations(self, raw):
        a = np.ascontiguousarray(raw)
        self._check(lib.mi_delbm_set_raw_populations(self.h, _ptr(a), a.nbytes))

    def get_raw_populations(self):
        dt = np.float32 if self.cfg.storage == STORE_F32 else np.uint16
        a = np.empty((19,) + self.shape, dtype=dt)
        self._check(lib.mi_delbm_get_raw_populations(self.h, _ptr(a), a.nbytes))
        return a

    def device_view(self):
        v = DeviceView()
        self._check(lib.mi_delbm_get_device_view(self.h, ctypes.byref(v)))
        return v

    # -- timing -----------------------------------------------------------
    def set_tuning(self, bulk_block_x=128, bulk_rows=1, bulk_pairs=False, list_blocks_per_sm=8):
        self._check(lib.mi_delbm_set_tuning(self.h, int(bulk_block_x), int(bulk_rows), int(bulk_pairs),
                                            int(list_blocks_per_sm)))

    def autotune(self, cache_path=None):
        bx, bl = c_int(0), c_int(0)
        self._check(lib.mi_delbm_autotune(self.h, cache_path.encode() if cache_path else None,
                                          ctypes.byref(bx), ctypes.byref(bl)))
        return self.get_tuning()

    def get_tuning(self):
        v = [c_int(0) for _ in range(4)]
        self._check(lib.mi_delbm_get_tuning(self.h, *[ctypes.byref(x) for x in v]))
        return {"bulk_block_x": v[0].value, "bulk_rows": v[1].value, "bulk_pairs": v[2].value,
                "list_blocks_per_sm": v[3].value}

    def set_schedule(self, overlap_boundary=False, unfused_dem=False, links_beside=False):
        """overlap_boundary: compute the boundary nodes beside the bulk kernel
        (True) or after it; unfused_dem: run DEM substeps as one launch
        sequence per substep instead of the fused substep kernel;
        links_beside: the links' bounce-back and momentum exchange beside the
        bulk kernel instead of after it."""
        flags = (SCHEDULE_OVERLAP_BOUNDARY if overlap_boundary else 0) | (SCHEDULE_UNFUSED_DEM if unfused_dem else 0) | \
            (SCHEDULE_LINKS_BESIDE if links_beside else 0)
        self._check(lib.mi_delbm_set_schedule(self.h, flags))

    def set_momentum_rules(self, cover_uncover=False):
        """cover_uncover: the momentum of nodes a particle covers or uncovers
        this step joins its hydrodynamic force and torque."""
        self._check(lib.mi_delbm_set_momentum_rules(self.h, MOMENTUM_COVER_UNCOVER if cover_uncover else 0))

    def set_graphs(self, on, device_loop=False):
        """on=False: individual launches; on=True: one graph per step, or with
        device_loop=True one graph launch per step() call (a conditional while
        node over two-step bodies)."""
        self._check(lib.mi_delbm_set_graphs(self.h, (2 if device_loop else 1) if on else 0))

    def set_timing(self, on):
        self._check(lib.mi_delbm_set_timing(self.h, 1 if on else 0))

    def phase_times(self, reset=True):
        ms = (c_double * 8)()
        n = (ctypes.c_longlong * 8)()
        self._check(lib.mi_delbm_phase_times(self.h, ms, n, 1 if reset else 0))
        return {PHASE_NAMES[b]: (ms[b], n[b]) for b in range(8)}

    def reserve_lists(self, boundary_nodes, links, new_nodes):
        self._check(lib.mi_delbm_reserve_lists(self.h, int(boundary_nodes), int(links), int(new_nodes)))

    def set_guess_wait(self, wait_rounds=0, stall=False):
        self._check(lib.mi_delbm_set_guess_wait(self.h, int(wait_rounds), 1 if stall else 0))

    def check(self):
        """mi_delbm_check: a dict of the counts; raises MiDelbmError (MI_ESTATE)
        when something is not finite."""
        hl = Health()
        st = lib.mi_delbm_check(self.h, ctypes.byref(hl))
        out = {f: getattr(hl, f) for f, _ in Health._fields_}
        if st != MI_OK:
            err = MiDelbmError(st, lib.mi_delbm_last_error(self.h).decode())
            err.health = out
            raise err
        return out

    def kernel_time(self, kernel):
        """(summed ms, launches) of one kernel's event-timed launches since the
        last phase_times reset."""
        ms, n = c_double(0.0), ctypes.c_longlong(0)
        self._check(lib.mi_delbm_kernel_time(self.h, kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def launch_count(self):
        return int(lib.mi_delbm_launch_count(self.h))

    # -- particles --------------------------------------------------------
    def add_particle(self, centers, k, density, skin, pos, quat, vel=(0, 0, 0), omega=(0, 0, 0), mass_props=None):
        c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
        kk = np.ascontiguousarray(k, dtype=np.float64).reshape(-1)
        vecs = [np.ascontiguousarray(v, dtype=np.float64) for v in (pos, quat, vel, omega)]
        mp = None
        if mass_props is not None:
            mp = MassProps()
            mp.mass = float(mass_props["mass"])
            mp.volume = float(mass_props["volume"])
            I = np.asarray(mass_props["inertia"], dtype=np.float64).reshape(9)
            for j in range(9):
                mp.inertia[j] = I[j]
        pid = c_int(-1)
        self._check(lib.mi_delbm_add_particle(self.h, len(kk), _ptr(c), _ptr(kk), float(density), float(skin),
                                              *[_ptr(v) for v in vecs],
                                              ctypes.byref(mp) if mp is not None else None, ctypes.byref(pid)))
        return pid.value

    def num_particles(self):
        return int(lib.mi_delbm_num_particles(self.h))

    def get_particle_state(self, pid):
        out = [np.zeros(3), np.zeros(4), np.zeros(3), np.zeros(3)]
        self._check(lib.mi_delbm_get_particle_state(self.h, int(pid), *[_ptr(v) for v in out]))
        return dict(zip(("pos", "quat", "vel", "omega"), out))

    def set_particle_state(self, pid, pos=None, quat=None, vel=None, omega=None):
        args = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in (pos, quat, vel, omega)]
        self._check(lib.mi_delbm_set_particle_state(self.h, int(pid), *[None if v is None else _ptr(v) for v in args]))

    def set_particle_states_ptr(self, ptr, n):
        """Queue an async upload of n x 13 doubles from host address ptr."""
        self._check(lib.mi_delbm_set_particle_states(self.h, c_void_p(int(ptr)), int(n)))

    def get_particle_states_ptr(self, ptr, n):
        """Queue an async download of n x 13 doubles to host address ptr."""
        self._check(lib.mi_delbm_get_particle_states(self.h, c_void_p(int(ptr)), int(n)))

    def forces_ptr(self, f_hydro, t_hydro):
        """Synchronising read of the hydrodynamic force/torque into host addresses."""
        self._check(lib.mi_delbm_forces(self.h, c_void_p(int(f_hydro)), c_void_p(int(t_hydro)), None, None))

    def get_particle_shape(self, pid):
        n = c_int(0)
        self._check(lib.mi_delbm_get_particle_shape(self.h, int(pid), None, None, 0, ctypes.byref(n), None, None))
        c = np.zeros((n.value, 3))
        k = np.zeros(n.value)
        mp = MassProps()
        rb = c_double(0)
        self._check(lib.mi_delbm_get_particle_shape(self.h, int(pid), _ptr(c), _ptr(k), n.value, ctypes.byref(n),
                                                    ctypes.byref(mp), ctypes.byref(rb)))
        return {"centers": c, "k": k, "mass": mp.mass, "volume": mp.volume,
                "inertia": np.array(mp.inertia[:]).reshape(3, 3), "Rb": rb.value}

    def forces(self):
        n = self.num_particles()
        out = [np.zeros((n, 3)) for _ in range(4)]
        self._check(lib.mi_delbm_forces(self.h, *[_ptr(v) for v in out]))
        return dict(zip(("F_hydro", "T_hydro", "F_contact", "T_contact"), out))

    def node_classes(self):
        cls = np.empty(self.shape, dtype=np.uint8)
        own = np.empty(self.shape, dtype=np.uint32)
        self._check(lib.mi_delbm_get_node_classes(self.h, _ptr(cls), _ptr(own), self.ncell))
        return cls, own

    def links(self):
        n = c_size_t(0)
        st = lib.mi_delbm_get_links(self.h, 0, None, None, None, None, ctypes.byref(n))
        if st not in (MI_OK, MI_ECAPACITY):
            self._check(st)
        m = n.value
        cell = np.empty(m, dtype=np.int32)
        d = np.empty(m, dtype=np.int8)
        p = np.empty(m, dtype=np.int32)
        q = np.empty(m, dtype=np.float32)
        self._check(lib.mi_delbm_get_links(self.h, m, _ptr(cell), _ptr(d), _ptr(p), _ptr(q), ctypes.byref(n)))
        return {"cell": cell, "dir": d, "particle": p, "q": q}

    def contacts(self):
        """Candidates of the last DEM substep as a list of dicts."""
        n = c_int(0)
        st = lib.mi_delbm_contacts(self.h, None, 0, ctypes.byref(n))
        if st not in (MI_OK, MI_ECAPACITY):
            self._check(st)
        arr = (Contact * max(1, n.value))()
        self._check(lib.mi_delbm_contacts(self.h, arr, n.value, ctypes.byref(n)))
        return [{"i": c.i, "j": c.j, "x_cp": np.array(c.xcp[:]), "n": np.array(c.n[:]), "delta": c.delta,
                 "iters": c.iters, "status": c.status} for c in arr[:n.value]]

    # -- learned guess -----------------------------------------------------
    def set_guess(self, mode, params=None):
        """GUESS_PLAIN, GUESS_WARM, or GUESS_LEARNED with the MLP parameters (float32 CUDA tensor)."""
        self._sync_in()
        self._check(lib.mi_delbm_set_guess(self.h, int(mode), _tp(params)))
        self._sync_out()

    def _sync_in(self):
        if self.torch_stream is not None:
            import torch
            self.torch_stream.wait_stream(torch.cuda.current_stream())

    def _sync_out(self):
        if self.torch_stream is not None:
            import torch
            torch.cuda.current_stream().wait_stream(self.torch_stream)
        else:
            self.synchronize()

    def pair_solve(self, ij, poses, flags, pred=None, X=None):
        """Closest points of explicitly posed pairs of this handle's particle
        shapes.  ij: (n, 2) int32 CUDA tensor, poses: (n, 14) float64 CUDA
        tensor; returns a dict of CUDA tensors (X, T, xm, iters, evals,
        status; those the flags produce)."""
        import torch
        n = int(ij.shape[0])
        dev = ij.device
        solve = bool(flags & (PAIR_PLAIN | PAIR_LEARNED))
        out = {}
        if flags & PAIR_FEATURES:
            X = torch.zeros((n, 64), dtype=torch.float32, device=dev)
        if X is not None:
            out["X"] = X
        if flags & PAIR_LABELS:
            out["T"] = torch.full((n, 4), float("nan"), dtype=torch.float32, device=dev)
        if solve:
            out["xm"] = torch.empty((n, 3), dtype=torch.float64, device=dev)
            for key in ("iters", "evals", "status"):
                out[key] = torch.empty(n, dtype=torch.int32, device=dev)
        self._sync_in()
        self._check(lib.mi_delbm_pair_solve(self.h, n, _tp(ij), _tp(poses), int(flags), _tp(pred), _tp(X),
                                            _tp(out.get("T")), _tp(out.get("xm")), _tp(out.get("iters")),
                                            _tp(out.get("evals")), _tp(out.get("status"))))
        self._sync_out()
        return out

    def stats(self):
        st = Stats()
        self._check(lib.mi_delbm_get_stats(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in Stats._fields_}


class CudaArray:
    """Minimal __cuda_array_interface__ wrapper so torch.as_tensor can view
    device memory owned by the library without copying."""

    def __init__(self, ptr, shape, typestr, strides=None, stream=None):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
            "version": 3, "strides": strides, "stream": None,
        }
