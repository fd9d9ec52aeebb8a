"""Helpers for the GPU parity tests: build/load the library, view device
buffers from torch, decode 16-bit storages.  Test plumbing only."""
import numpy as np

_built = False


def binding():
    global _built
    if not _built:
        from paper_2209_10411_gb300 import build
        build.build()
        _built = True
    from paper_2209_10411_gb300 import _binding
    return _binding


def pop_tensor(sim):
    """torch view (19, plane_stride) of the current stored populations."""
    import torch
    B = binding()
    sim.synchronize()
    v = sim.device_view()
    typestr = "<f4" if v.storage == B.STORE_F32 else "<i2"
    arr = B.CudaArray(v.populations, (19, v.plane_stride), typestr)
    return torch.as_tensor(arr, device="cuda")


class DeviceGather:
    """Indexable as g[i, z, y, x] (integer arrays) returning float64 numpy
    populations gathered on the device; used to feed the oracle sampled inputs
    of lattices too large to copy."""

    def __init__(self, sim):
        import torch
        sim.synchronize()
        self.t = pop_tensor(sim)
        self.nz, self.ny, self.nx = sim.shape
        self.shape = (19, self.nz, self.ny, self.nx)
        self.storage = sim.cfg.storage
        self.torch = torch

    def __getitem__(self, idx):
        i, z, y, x = idx
        torch = self.torch
        lin = (np.asarray(z, dtype=np.int64) * self.ny + np.asarray(y, dtype=np.int64)) * self.nx \
            + np.asarray(x, dtype=np.int64)
        li = torch.as_tensor(lin, device="cuda")
        vals = self.t[int(i)].index_select(0, li)
        from oracle.d3q19 import W
        if self.storage == 0:
            return vals.cpu().numpy().astype(np.float64)
        raw = vals.cpu().numpy()
        return decode(raw, self.storage) + W[int(i)]


def decode(raw, storage):
    """Exact float64 value of stored 16-bit deviations."""
    raw = np.asarray(raw)
    if storage == 1:
        return raw.view(np.uint16).view(np.float16).astype(np.float64)
    if storage == 2:
        u = raw.view(np.uint16).astype(np.uint32) << 16
        return u.view(np.float32).astype(np.float64)
    return raw.astype(np.float64)


def ulp16(x, storage):
    """One unit in the last place of the 16-bit storage at |x|."""
    mant = 10 if storage == 1 else 7
    min_exp = -14 if storage == 1 else -126
    e = np.floor(np.log2(np.maximum(np.abs(x), 1e-300)))
    e = np.maximum(e, min_exp)
    return np.exp2(e - mant)
