"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/mi_delbm.h declares (no compute call: this runs on CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(mi_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_10411_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ["mi_delbm_create", "mi_delbm_destroy", "mi_delbm_step", "mi_delbm_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, "declared in include/ but not exported: %s" % missing


def test_config_layout_matches_binding(lib):
    from paper_2209_10411_gb300 import _binding as B
    assert B.lib.mi_delbm_abi_version() == 2
    assert B.lib.mi_delbm_config_size() == ctypes.sizeof(B.Config)
    cfg = B.Config()
    B.lib.mi_delbm_config_init(ctypes.byref(cfg))
    assert (cfg.nx, cfg.ny, cfg.nz) == (64, 64, 64)
    assert abs(cfg.tau - 0.8) < 1e-15 and cfg.dem_substeps == 1
    assert cfg.storage == B.STORE_F32 and cfg.bb_mode == B.BB_IBB


def test_create_rejects_bad_config_without_touching_gpu(lib):
    from paper_2209_10411_gb300 import _binding as B
    cfg = B.Config()
    B.lib.mi_delbm_config_init(ctypes.byref(cfg))
    cfg.tau = 0.5
    h = ctypes.c_void_p()
    st = B.lib.mi_delbm_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == B.MI_EINVAL and not h.value
    assert b"tau" in B.lib.mi_delbm_last_error(None)
    B.lib.mi_delbm_config_init(ctypes.byref(cfg))
    cfg.nx = 0
    assert B.lib.mi_delbm_create(ctypes.byref(cfg), ctypes.byref(h)) == B.MI_EINVAL


def test_fitting_and_shape_entry_points_validate_on_host(lib):
    """Argument checks of mi_gs_fit, mi_ga_run and mi_shape_descriptors come
    before any CUDA call: bad sizes or parameters return MI_EINVAL, empty
    batches MI_OK, both without a GPU."""
    from paper_2209_10411_gb300 import _binding as B
    L = B.lib
    N = None
    # Gradient Search: negative batch, point/ball limits, non-finite step
    assert L.mi_gs_fit(-1, N, N, N, N, N, N, 16, 8, 10, 0.1, N, N, N) == B.MI_EINVAL
    assert L.mi_gs_fit(1, N, N, N, N, N, N, 10241, 8, 10, 0.1, N, N, N) == B.MI_EINVAL
    assert L.mi_gs_fit(1, N, N, N, N, N, N, 16, 257, 10, 0.1, N, N, N) == B.MI_EINVAL
    assert L.mi_gs_fit(1, N, N, N, N, N, N, 16, 8, 10, float("nan"), N, N, N) == B.MI_EINVAL
    assert L.mi_gs_fit(1, N, N, N, N, N, N, 16, 8, 10, 0.1, N, N, N) == B.MI_EINVAL   # NULL arrays
    assert L.mi_gs_fit(0, N, N, N, N, N, N, 16, 8, 10, 0.1, N, N, N) == B.MI_OK
    # Genetic Algorithm: population of one, rates outside [0, 1], NULL arrays
    args = [N, 64, N, 10, N, N, 0.1, 0.5, 1, 5, 1, N, N, N, N, N, N]
    assert L.mi_ga_run(1, 4, *args) == B.MI_EINVAL
    bad_cm = list(args)
    bad_cm[6] = 1.5
    assert L.mi_ga_run(8, 4, *bad_cm) == B.MI_EINVAL
    assert L.mi_ga_run(8, 4, *args) == B.MI_EINVAL
    assert L.mi_ga_scratch_bytes(0, 4) == 0 and L.mi_ga_scratch_bytes(8, 4) > 0
    # shape descriptors: spacing, band width
    assert L.mi_shape_descriptors(1, N, N, N, N, 8, 0.0, 0.1, N, N, N, N) == B.MI_EINVAL
    assert L.mi_shape_descriptors(1, N, N, N, N, 8, 0.1, 1.0, N, N, N, N) == B.MI_EINVAL
    assert L.mi_shape_descriptors(1, N, N, N, N, 0, 0.1, 0.1, N, N, N, N) == B.MI_EINVAL
    assert L.mi_shape_descriptors(1, N, N, N, N, 8, 0.1, 0.1, N, N, N, N) == B.MI_EINVAL  # NULL arrays
    assert L.mi_shape_descriptors(0, N, N, N, N, 8, 0.1, 0.1, N, N, N, N) == B.MI_OK
    assert L.mi_shape_scratch_bytes(0, 8) == 0 and L.mi_shape_scratch_bytes(2, 8) > 0


def test_create_validates_every_config_field_on_host(lib):
    """Each invalid field of mi_delbm_config is refused with MI_EINVAL and a
    message naming it, before any CUDA call."""
    from paper_2209_10411_gb300 import _binding as B
    cases = [("nx", 0, b"lattice sizes"), ("nz", 70000, b"lattice sizes"), ("rho0", 0.0, b"rho0"),
             ("storage", 3, b"storage"), ("bb_mode", 7, b"bb_mode"), ("dem_substeps", 0, b"dem_substeps"),
             ("max_particles", 70000, b"max_particles"), ("max_balls", -1, b"capacities"),
             ("guess_mode", B.GUESS_LEARNED, b"guess_mode")]
    for field, value, msg in cases:
        cfg = B.Config()
        B.lib.mi_delbm_config_init(ctypes.byref(cfg))
        setattr(cfg, field, value)
        h = ctypes.c_void_p()
        assert B.lib.mi_delbm_create(ctypes.byref(cfg), ctypes.byref(h)) == B.MI_EINVAL, field
        assert not h.value
        assert msg in B.lib.mi_delbm_last_error(None), (field, B.lib.mi_delbm_last_error(None))
    cfg = B.Config()
    B.lib.mi_delbm_config_init(ctypes.byref(cfg))
    cfg.nx, cfg.ny, cfg.nz = 2048, 2048, 1024          # 2^32 nodes
    h = ctypes.c_void_p()
    assert B.lib.mi_delbm_create(ctypes.byref(cfg), ctypes.byref(h)) == B.MI_EINVAL
    assert b"2^31-1" in B.lib.mi_delbm_last_error(None)
