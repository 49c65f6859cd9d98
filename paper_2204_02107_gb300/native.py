"""ctypes binding of ``libventflow.so`` (declared in ``include/ventflow.h``): argument marshalling only.

Every computation runs in the library's CUDA kernels.  If the library has not been built, every entry point
raises ``VentflowUnavailable``; there is no CPU fallback.

Host arrays are numpy arrays (C-contiguous, the dtype the call needs); device arrays are CUDA torch tensors,
passed by pointer.  Shapes follow the library layout: (nz, ny, nx), x fastest.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libventflow.so")

VF_OK, VF_EINVAL, VF_ESIZE, VF_ENOMEM, VF_ECUDA, VF_ESTATE, VF_ENONFINITE, VF_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
VF_FP64, VF_FP32_MIXED = 0, 1
VF_HOST, VF_DEVICE = 0, 1
FIELDS = {"u": 0, "v": 1, "w": 2, "c": 3, "p": 4}
N_PHASES = 17
PRECISIONS = {"fp64": VF_FP64, "fp32": VF_FP32_MIXED, "fp32_mixed": VF_FP32_MIXED}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class VfAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class VfGridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("nu", C.c_double), ("alpha_c", C.c_double), ("dt", C.c_double), ("tau_f", C.c_double),
                ("body_force", C.c_double * 3),
                ("n_pressure_iters", C.c_int32), ("filter", C.c_int32), ("precision", C.c_int32),
                ("history_capacity", C.c_int32),
                ("cuda_stream", C.c_void_p), ("alloc", C.POINTER(VfAllocator)), ("courant_max", C.c_double)]


class VfBatchDesc(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("reduce_every", C.c_int32),
                ("cuda_stream", C.c_void_p), ("autotune", C.c_int32)]


class VfTiles(C.Structure):
    _fields_ = [("zc_stage", C.c_int32), ("zc_div", C.c_int32), ("zc_project", C.c_int32),
                ("zc_filter", C.c_int32), ("fft_x", C.c_int32), ("fft_y", C.c_int32), ("fft_z", C.c_int32)]

    def to_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class VfReduce(C.Structure):
    _fields_ = [("t", C.c_double), ("step", C.c_int64), ("ke", C.c_double), ("div_max", C.c_double),
                ("div_l2", C.c_double), ("u_max", C.c_double), ("c_total", C.c_double), ("c_room", C.c_double),
                ("c2_room", C.c_double), ("v_room", C.c_double), ("hist", C.c_int64 * 64),
                ("hist_under", C.c_int64), ("hist_over", C.c_int64), ("dt", C.c_double),
                ("budget_forcing", C.c_double), ("budget_forcing_room", C.c_double),
                ("budget_outflow", C.c_double), ("budget_mask_loss", C.c_double),
                ("budget_filter_room", C.c_double)]

    def to_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "hist"}
        d["hist"] = np.array(self.hist[:], dtype=np.int64)
        return d


class VentflowUnavailable(RuntimeError):
    pass


class VentflowError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{status_string(code)} ({code}): {message}")
        self.code = code


_lib = None

_SIGNATURES = {
    "vf_grid_desc_default": (C.c_int, [C.POINTER(VfGridDesc)]),
    "vf_create_grid": (C.c_int, [C.POINTER(VfGridDesc), C.POINTER(C.c_void_p)]),
    "vf_destroy": (C.c_int, [C.c_void_p]),
    "vf_set_mask": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "vf_set_inflow": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_int]),
    "vf_set_region": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "vf_set_inflow_tanh": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double]),
    "vf_set_inflow_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_double,
                                       C.c_int]),
    "vf_set_field": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "vf_set_time": (C.c_int, [C.c_void_p, C.c_double, C.c_int64]),
    "vf_step": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32]),
    "vf_sync": (C.c_int, [C.c_void_p]),
    "vf_read_field": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "vf_reductions": (C.c_int, [C.c_void_p, C.POINTER(VfReduce)]),
    "vf_history": (C.c_int, [C.c_void_p, C.POINTER(VfReduce), C.c_int64, C.POINTER(C.c_int64)]),
    "vf_clear_history": (C.c_int, [C.c_void_p]),
    "vf_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                          C.POINTER(C.c_int64)]),
    "vf_poisson_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vf_grid_bytes": (C.c_int64, [C.POINTER(VfGridDesc)]),
    "vf_get_tiles": (C.c_int, [C.c_void_p, C.POINTER(VfTiles)]),
    "vf_fft_path": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "vf_set_tiles": (C.c_int, [C.c_void_p, C.POINTER(VfTiles)]),
    "vf_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(VfTiles)]),
    "vf_fft_schedules": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    "vf_tile_cache_size": (C.c_int64, []),
    "vf_tile_cache_entry": (C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.POINTER(VfTiles)]),
    "vf_tile_cache_insert": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(VfTiles)]),
    "vf_tile_cache_lookup": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(VfTiles)]),
    "vf_tile_cache_clear": (C.c_int, []),
    "vf_batch_create": (C.c_int, [C.POINTER(VfBatchDesc), C.POINTER(C.c_void_p)]),
    "vf_batch_destroy": (C.c_int, [C.c_void_p]),
    "vf_batch_add": (C.c_int, [C.c_void_p, C.POINTER(VfGridDesc), C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_double), C.c_double, C.c_void_p, C.c_int, C.c_int64, C.c_int,
                               C.POINTER(C.c_int32)]),
    "vf_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "vf_batch_sync": (C.c_int, [C.c_void_p]),
    "vf_batch_poll": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
    "vf_batch_grid": (C.c_void_p, [C.c_void_p, C.c_int32]),
    "vf_batch_remove": (C.c_int, [C.c_void_p, C.c_int32]),
    "vf_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
    "vf_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "vf_poisson_solve_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                           C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vf_poisson_noalloc_max_cells": (C.c_int64, [C.c_int32]),
    "vf_profile_steps": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64)]),
    "vf_phase_name": (C.c_char_p, [C.c_int]),
    "vf_status_string": (C.c_char_p, [C.c_int]),
    "vf_abi_sizes": (C.c_int, [C.POINTER(C.c_int64)]),
    "vf_measure_fp64_rate": (C.c_int, [C.POINTER(C.c_double)]),
    "vf_set_inflow_field": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "vf_set_force_region": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "vf_region_force": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "vf_particles_set": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                   C.c_double, C.POINTER(C.c_double)]),
    "vf_particles_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vf_particles_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "vf_last_error": (C.c_char_p, [C.c_void_p]),
    "vf_ach_log_slope": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64,
                                   C.POINTER(C.c_double)]),
    "vf_ach_fit3": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "vf_wells_riley": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
}


def lib():
    """The loaded library (loads it on first use)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise VentflowUnavailable(f"{LIB_PATH} is not built; run paper_2204_02107_gb300.build.build()")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def status_string(code):
    return lib().vf_status_string(int(code)).decode()


def _dptr(arr):
    return C.cast(arr.ctypes.data, C.POINTER(C.c_double))


def _is_tensor(x):
    return type(x).__module__.startswith("torch")


def _device_tensor(x, dtypes, n, what):
    """Check that x is a contiguous CUDA tensor whose dtype name is in ``dtypes`` ('float64', 'float32',
    'uint8') with n elements (n None: any count) before its address goes to the library, which would otherwise
    read past a smaller buffer or through a host pointer."""
    if not _is_tensor(x) or not x.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    name = str(x.dtype).replace("torch.", "")
    if name not in dtypes:
        raise TypeError(f"{what}: dtype {name} not one of {', '.join(dtypes)}")
    if not x.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if n is not None and x.numel() != n:
        raise ValueError(f"{what}: expected {n} elements, got {x.numel()}")
    return x


def _pointer(x, dtype, n):
    """(pointer, mem, keepalive) for a numpy array (host) or CUDA torch tensor (device) of n values; a device
    tensor must hold elements of ``dtype`` (None: float64 or float32)."""
    if _is_tensor(x):
        if not x.is_cuda:
            x = x.detach().cpu().numpy()
        else:
            want = ("float64", "float32") if dtype is None else (np.dtype(dtype).name,)
            _device_tensor(x, want, n, "device array")
            return C.c_void_p(x.data_ptr()), VF_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    if a.size != n:
        raise ValueError(f"array must have {n} elements, got {a.size}")
    return C.c_void_p(a.ctypes.data), VF_HOST, a


def default_desc():
    d = VfGridDesc()
    lib().vf_grid_desc_default(C.byref(d))
    return d


def make_desc(nx, ny, nz, lx, ly, lz, nu, dt, alpha_c=None, tau_f=0.0, body_force=(0.0, 0.0, 0.0),
              n_pressure_iters=4, filter=True, precision="fp32", history_capacity=4096, stream=None,
              courant_max=0.0):
    d = default_desc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.lx, d.ly, d.lz = lx, ly, lz
    d.nu = nu
    d.alpha_c = -1.0 if alpha_c is None else alpha_c
    d.dt = dt
    d.tau_f = tau_f
    for j in range(3):
        d.body_force[j] = body_force[j]
    d.n_pressure_iters = n_pressure_iters
    d.filter = 1 if filter else 0
    d.precision = PRECISIONS[precision]
    d.history_capacity = history_capacity
    d.cuda_stream = C.c_void_p(stream) if stream else None
    d.courant_max = courant_max
    return d


def room_desc(room, precision="fp32", filter=True, n_pressure_iters=4, nu=1.6e-5, dt=None, **kw):
    """Grid description of a ``rooms.Room``."""
    return make_desc(room.nx, room.ny, room.nz, room.lx, room.ly, room.lz, nu, room.dt if dt is None else dt,
                     filter=filter, n_pressure_iters=n_pressure_iters, precision=precision, **kw)


def grid_bytes(desc):
    return int(lib().vf_grid_bytes(C.byref(desc)))


class Batch:
    """Rooms of uneven size advanced together (vf_batch_*): one CUDA graph launch per batch step, one branch per
    room.  Slots are admitted against ``hbm_budget_bytes``."""

    def __init__(self, max_slots, hbm_budget_bytes, reduce_every=1, stream=None, autotune=0):
        d = VfBatchDesc(max_slots, int(hbm_budget_bytes), reduce_every, C.c_void_p(stream) if stream else None,
                        int(autotune))
        h = C.c_void_p()
        rc = lib().vf_batch_create(C.byref(d), C.byref(h))
        if rc != VF_OK:
            raise VentflowError(rc, "vf_batch_create")
        self._h = h
        self.max_slots = max_slots
        self._desc = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().vf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != VF_OK:
            msg = lib().vf_batch_last_error(self._h)
            raise VentflowError(rc, f"{what}: {msg.decode() if msg else ''}")

    def add(self, desc, beta, S, u_set, c_set, steps, room=None, c0=None):
        """Admit a room; returns its slot.  Raises VentflowError(VF_ENOMEM) when it does not fit."""
        n = desc.nx * desc.ny * desc.nz
        pb, mem, kb = _pointer(beta, np.uint8, n)
        ps = _pointer(S, np.uint8, n) if S is not None else (None, mem, None)
        pr = _pointer(room, np.uint8, n) if room is not None else (None, mem, None)
        c0_is64 = True   # float32 values (host or device) pass as they are, anything else as float64
        if c0 is None:
            pc = (None, mem, None)
        elif _is_tensor(c0) and c0.is_cuda:
            import torch
            c0_is64 = c0.dtype != torch.float32
            pc = _pointer(c0, np.float64 if c0_is64 else np.float32, n)
        else:
            c0 = np.asarray(c0)
            c0_is64 = c0.dtype != np.float32
            pc = _pointer(c0, np.float64 if c0_is64 else np.float32, n)
        if len({p[1] for p in (ps, pr, pc)} | {mem}) != 1:
            raise ValueError("beta, S, room and c0 must all be host arrays or all CUDA tensors")
        us = (C.c_double * 3)(*u_set)
        slot = C.c_int32()
        rc = lib().vf_batch_add(self._h, C.byref(desc), pb, ps[0], pr[0], us, float(c_set), pc[0],
                                1 if c0_is64 else 0, int(steps), mem, C.byref(slot))
        self._check(rc, "vf_batch_add")
        self._desc[slot.value] = desc
        return slot.value

    def step(self, n):
        self._check(lib().vf_batch_step(self._h, int(n)), "vf_batch_step")

    def sync(self):
        self._check(lib().vf_batch_sync(self._h), "vf_batch_sync")

    def poll(self):
        buf = (C.c_int32 * self.max_slots)()
        n = C.c_int32()
        self._check(lib().vf_batch_poll(self._h, buf, self.max_slots, C.byref(n)), "vf_batch_poll")
        return [buf[i] for i in range(min(n.value, self.max_slots))]

    def grid(self, slot):
        """Borrowed Grid of a slot (valid until the slot is removed)."""
        h = lib().vf_batch_grid(self._h, int(slot))
        if not h:
            raise VentflowError(VF_EINVAL, f"slot {slot} is empty")
        return Grid.borrowed(h, self._desc[slot])

    def remove(self, slot):
        self._check(lib().vf_batch_remove(self._h, int(slot)), "vf_batch_remove")
        self._desc.pop(slot, None)

    def info(self):
        a, dn, b, s = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
        self._check(lib().vf_batch_info(self._h, C.byref(a), C.byref(dn), C.byref(b), C.byref(s)), "vf_batch_info")
        return dict(active=a.value, done=dn.value, bytes_in_use=b.value, batch_steps=s.value)


class Grid:
    """One room grid on the current CUDA device (``vf_create_grid``).  Sizes (nx, ny, nz) must be even, >= 8 and
    2-3-5 smooth.  ``precision`` is 'fp64' or 'fp32' (FP32 fields, FP64 reductions)."""

    def __init__(self, nx, ny, nz, lx, ly, lz, nu, dt, alpha_c=None, tau_f=0.0, body_force=(0.0, 0.0, 0.0),
                 n_pressure_iters=4, filter=True, precision="fp32", history_capacity=4096, stream=None,
                 courant_max=0.0):
        d = make_desc(nx, ny, nz, lx, ly, lz, nu, dt, alpha_c, tau_f, body_force, n_pressure_iters, filter,
                      precision, history_capacity, stream, courant_max)
        h = C.c_void_p()
        rc = lib().vf_create_grid(C.byref(d), C.byref(h))
        if rc != VF_OK:
            raise VentflowError(rc, "vf_create_grid")
        self._owned = True
        self._h = h
        self.desc = d
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.precision = precision

    @classmethod
    def borrowed(cls, handle, desc):
        """A view of a grid owned by someone else (a batch slot): never destroyed by this object."""
        g = cls.__new__(cls)
        g._owned = False
        g._h = C.c_void_p(handle)
        g.desc = desc
        g.shape = (desc.nz, desc.ny, desc.nx)
        g.n = desc.nx * desc.ny * desc.nz
        g.precision = "fp64" if desc.precision == VF_FP64 else "fp32"
        return g

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                lib().vf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, what):
        if rc != VF_OK:
            msg = lib().vf_last_error(self._h)
            raise VentflowError(rc, f"{what}: {msg.decode() if msg else ''}")

    # -- inputs
    def set_mask(self, beta):
        ptr, mem, _keep = _pointer(beta, np.uint8, self.n)
        self._check(lib().vf_set_mask(self._h, ptr, mem), "vf_set_mask")

    def set_inflow(self, S, u_set, c_set):
        us = (C.c_double * 3)(*u_set)
        if S is None:
            self._check(lib().vf_set_inflow(self._h, None, us, float(c_set), VF_HOST), "vf_set_inflow")
            return
        ptr, mem, _keep = _pointer(S, np.uint8, self.n)
        self._check(lib().vf_set_inflow(self._h, ptr, us, float(c_set), mem), "vf_set_inflow")

    def set_inflow_tanh(self, center, width, sharpness, u_set, c_set):
        """Smooth forcing window of Eq. 5 (centre, width [m] and sharpness B per axis x, y, z)."""
        d3 = lambda v: (C.c_double * 3)(*[float(a) for a in v])
        self._check(lib().vf_set_inflow_tanh(self._h, d3(center), d3(width), d3(sharpness), d3(u_set),
                                             float(c_set)), "vf_set_inflow_tanh")

    def set_inflow_values(self, S, u_set, c_set):
        """Smooth forcing region from values in [0, 1] (float64 numpy array or CUDA tensor of the grid's size)."""
        is64 = True
        if _is_tensor(S) and S.is_cuda:
            import torch
            is64 = S.dtype == torch.float64
            ptr, mem, _keep = _pointer(S, None, self.n)
        else:
            ptr, mem, _keep = _pointer(S, np.float64, self.n)
        us = (C.c_double * 3)(*u_set)
        self._check(lib().vf_set_inflow_values(self._h, ptr, 1 if is64 else 0, us, float(c_set), mem),
                    "vf_set_inflow_values")

    def set_particles(self, pos, vel, size, rho_p=1000.0, rho_f=1.2, gravity=(0.0, 0.0, -9.81)):
        """Lagrangian particles: pos, vel (n, 3) [m], [m/s]; size (n,) d [m]."""
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        size = np.ascontiguousarray(size, dtype=np.float64).reshape(-1)
        n = pos.shape[0]
        if vel.shape[0] != n or size.shape[0] != n:
            raise ValueError("pos, vel and size must describe the same particles")
        g3 = (C.c_double * 3)(*gravity)
        self._check(lib().vf_particles_set(self._h, n, C.c_void_p(pos.ctypes.data), C.c_void_p(vel.ctypes.data),
                                           C.c_void_p(size.ctypes.data), float(rho_p), float(rho_f), g3),
                    "vf_particles_set")

    def particles(self):
        """(pos (n, 3), vel (n, 3), deposited (n,) bool) after the enqueued steps."""
        n = C.c_int64()
        self._check(lib().vf_particles_count(self._h, C.byref(n)), "vf_particles_count")
        pos = np.zeros((n.value, 3))
        vel = np.zeros((n.value, 3))
        dep = np.zeros(n.value, dtype=np.int32)
        if n.value:
            self._check(lib().vf_particles_read(self._h, C.c_void_p(pos.ctypes.data), C.c_void_p(vel.ctypes.data),
                                                C.c_void_p(dep.ctypes.data)), "vf_particles_read")
        return pos, vel, dep.astype(bool)

    def set_inflow_field(self, S, targets):
        """Forcing with per-cell targets: S (grid-sized) and targets (4 grid-sized arrays u, v, w, c), float64."""
        Sa = np.ascontiguousarray(S, dtype=np.float64).reshape(-1)
        Ta = np.ascontiguousarray(np.stack([np.asarray(t, dtype=np.float64).reshape(-1) for t in targets]))
        if Sa.size != self.n or Ta.shape != (4, self.n):
            raise ValueError("S must have one value per cell and targets four arrays of the grid's size")
        self._check(lib().vf_set_inflow_field(self._h, C.c_void_p(Sa.ctypes.data), C.c_void_p(Ta.ctypes.data), 1,
                                              VF_HOST), "vf_set_inflow_field")

    def set_force_region(self, region):
        ptr, mem, _keep = _pointer(region, np.uint8, self.n)
        self._check(lib().vf_set_force_region(self._h, ptr, mem), "vf_set_force_region")

    def region_force(self):
        f = (C.c_double * 3)()
        self._check(lib().vf_region_force(self._h, f), "vf_region_force")
        return tuple(f)

    def set_region(self, room):
        ptr, mem, _keep = _pointer(room, np.uint8, self.n)
        self._check(lib().vf_set_region(self._h, ptr, mem), "vf_set_region")

    def set_field(self, name, values):
        if _is_tensor(values) and values.is_cuda:
            import torch
            is64 = values.dtype == torch.float64
            ptr, mem, _keep = _pointer(values, None, self.n)
        else:
            arr = np.asarray(values)
            is64 = arr.dtype != np.float32
            ptr, mem, _keep = _pointer(arr, np.float64 if is64 else np.float32, self.n)
        self._check(lib().vf_set_field(self._h, FIELDS[name], ptr, 1 if is64 else 0, mem), "vf_set_field")

    def set_time(self, t, step):
        self._check(lib().vf_set_time(self._h, float(t), int(step)), "vf_set_time")

    # -- stepping
    def step(self, n=1, reduce_every=0):
        self._check(lib().vf_step(self._h, int(n), int(reduce_every)), "vf_step")

    def sync(self):
        self._check(lib().vf_sync(self._h), "vf_sync")

    # -- outputs
    def read_field(self, name, as_fp64=True):
        out = np.empty(self.shape, dtype=np.float64 if as_fp64 else np.float32)
        self._check(lib().vf_read_field(self._h, FIELDS[name], C.c_void_p(out.ctypes.data), 1 if as_fp64 else 0,
                                        VF_HOST), "vf_read_field")
        return out

    def read_field_into(self, name, tensor):
        """Device-to-device read into a contiguous CUDA tensor (float64 or float32)."""
        import torch
        _device_tensor(tensor, ("float64", "float32"), self.n, "read_field_into")
        ptr, mem, _keep = _pointer(tensor, None, self.n)
        self._check(lib().vf_read_field(self._h, FIELDS[name], ptr, 1 if tensor.dtype == torch.float64 else 0, mem),
                    "vf_read_field")

    def reductions(self):
        r = VfReduce()
        self._check(lib().vf_reductions(self._h, C.byref(r)), "vf_reductions")
        return r.to_dict()

    def history(self, max_records=None):
        if max_records is None:
            max_records = self.desc.history_capacity
        buf = (VfReduce * max(1, max_records))()
        count = C.c_int64()
        self._check(lib().vf_history(self._h, buf, int(max_records), C.byref(count)), "vf_history")
        return [buf[i].to_dict() for i in range(count.value)]

    def clear_history(self):
        self._check(lib().vf_clear_history(self._h), "vf_clear_history")

    def info(self):
        t, s, cells, nbytes = C.c_double(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(lib().vf_info(self._h, C.byref(t), C.byref(s), C.byref(cells), C.byref(nbytes)), "vf_info")
        return dict(t=t.value, step=s.value, cells=cells.value, device_bytes=nbytes.value)

    def profile_steps(self, n, reduce_every=0):
        """n steps with CUDA events after every launch: {phase name: (total ms, launches)}."""
        ms = (C.c_double * N_PHASES)()
        cnt = (C.c_int64 * N_PHASES)()
        self._check(lib().vf_profile_steps(self._h, int(n), int(reduce_every), ms, cnt), "vf_profile_steps")
        return {lib().vf_phase_name(i).decode(): (ms[i], cnt[i]) for i in range(N_PHASES) if cnt[i] > 0}

    def tiles(self):
        """The launch tiles of this grid: z-chunks per kernel family and the FFT radix schedule per axis."""
        t = VfTiles()
        self._check(lib().vf_get_tiles(self._h, C.byref(t)), "vf_get_tiles")
        return t.to_dict()

    def fft_path(self):
        """'generic', 'register_plane' or 'register_tile': the passes of this grid's pressure solve."""
        p = C.c_int32()
        self._check(lib().vf_fft_path(self._h, C.byref(p)), "vf_fft_path")
        return ("generic", "register_plane", "register_tile")[p.value]

    def set_tiles(self, zc_stage, zc_div, zc_project, zc_filter, fft_x=None, fft_y=None, fft_z=None):
        """Set the z-chunks; FFT schedule indices left as None keep the grid's current ones."""
        cur = self.tiles()
        fft = [cur[k] if v is None else v for k, v in (("fft_x", fft_x), ("fft_y", fft_y), ("fft_z", fft_z))]
        t = VfTiles(zc_stage, zc_div, zc_project, zc_filter, *fft)
        self._check(lib().vf_set_tiles(self._h, C.byref(t)), "vf_set_tiles")

    def autotune(self, reps=5):
        """Time every z-chunk per kernel family on this grid, then (generic FFT path) every radix schedule per
        axis; keep the fastest and cache them for the shape."""
        t = VfTiles()
        self._check(lib().vf_autotune(self._h, int(reps), C.byref(t)), "vf_autotune")
        return t.to_dict()

    def poisson_solve(self, f, p):
        """Solve L p = f on the device (f, p: contiguous CUDA tensors in the grid's precision)."""
        want = ("float64",) if self.precision == "fp64" else ("float32",)
        _device_tensor(f, want, self.n, "poisson_solve f")
        _device_tensor(p, want, self.n, "poisson_solve p")
        self._check(lib().vf_poisson_solve(self._h, C.c_void_p(f.data_ptr()), C.c_void_p(p.data_ptr())),
                    "vf_poisson_solve")


def fft_schedules(n):
    """Candidate radix schedules of the generic FFT passes for length n (``vf_fft_schedules``), default first."""
    out = []
    buf = (C.c_int32 * 16)()
    while True:
        k = lib().vf_fft_schedules(int(n), len(out), buf, 16)
        if k < 0:
            raise VentflowError(k, "vf_fft_schedules")
        if k == 0:
            return out
        out.append([buf[i] for i in range(k)])


def measure_fp64_rate():
    """FP64 FMA rate of the current device [GFLOP/s]."""
    v = C.c_double()
    rc = lib().vf_measure_fp64_rate(C.byref(v))
    if rc != VF_OK:
        raise VentflowError(rc, "vf_measure_fp64_rate")
    return v.value


def tile_cache_lookup(nx, ny, nz, precision="fp32"):
    """The cached tiles of a shape, or None."""
    t = VfTiles()
    prec = VF_FP64 if precision == "fp64" else VF_FP32_MIXED
    return t.to_dict() if lib().vf_tile_cache_lookup(nx, ny, nz, prec, C.byref(t)) == 1 else None


def tile_cache_clear():
    lib().vf_tile_cache_clear()


def tile_cache_entries():
    """Every tile-cache entry: a list of ((nx, ny, nz, 'fp64' | 'fp32'), tiles dict) in key order."""
    out = []
    key = (C.c_int32 * 4)()
    for i in range(int(lib().vf_tile_cache_size())):
        t = VfTiles()
        rc = lib().vf_tile_cache_entry(i, key, C.byref(t))
        if rc != VF_OK:
            raise VentflowError(rc, "vf_tile_cache_entry")
        out.append(((key[0], key[1], key[2], "fp64" if key[3] == VF_FP64 else "fp32"), t.to_dict()))
    return out


def tile_cache_insert(nx, ny, nz, precision, tiles):
    """Store tiles (a dict with the vf_tiles fields) for a shape and precision, as the autotuner does."""
    t = VfTiles(**{name: int(tiles[name]) for name, _ in VfTiles._fields_})
    rc = lib().vf_tile_cache_insert(int(nx), int(ny), int(nz), PRECISIONS[precision], C.byref(t))
    if rc != VF_OK:
        raise VentflowError(rc, "vf_tile_cache_insert")


def tile_cache_save(path):
    """Write the tile cache to a JSON file (a list of {"nx", "ny", "nz", "precision", "tiles"})."""
    import json
    entries = [{"nx": k[0], "ny": k[1], "nz": k[2], "precision": k[3], "tiles": t} for k, t in tile_cache_entries()]
    with open(path, "w") as f:
        json.dump(entries, f, indent=1)


def tile_cache_load(path):
    """Add the entries of a JSON file written by tile_cache_save to the tile cache (each checked by the library);
    returns the number loaded."""
    import json
    with open(path) as f:
        entries = json.load(f)
    for e in entries:
        tile_cache_insert(e["nx"], e["ny"], e["nz"], e["precision"], e["tiles"])
    return len(entries)


def _noalloc_sizes_accepted(nx, ny, nz, precision):
    """The size rules vf_poisson_solve_noalloc states: even, >= 8, 2-3-5 smooth, at most its cell limit, every FFT
    length (nx/2 + 1, ny, nz) at most 1024, ny and nz at most 581 (FP64) or 592 (FP32)."""
    def smooth(n):
        if n < 8 or n % 2:
            return False
        for q in (2, 3, 5):
            while n % q == 0:
                n //= q
        return n == 1
    yz_max = 581 if precision == VF_FP64 else 592
    return (all(smooth(int(v)) for v in (nx, ny, nz)) and nx * ny * nz <= lib().vf_poisson_noalloc_max_cells(precision)
            and max(nx // 2 + 1, ny, nz) <= 1024 and max(ny, nz) <= yz_max)


def poisson_solve_noalloc(nx, ny, nz, lx, ly, lz, f, p, stream=None):
    """Solve L p = f without any device allocation (f, p: contiguous CUDA tensors, float64 or float32)."""
    _device_tensor(f, ("float64", "float32"), None, "poisson_solve_noalloc f")
    dt = str(f.dtype).replace("torch.", "")
    _device_tensor(p, (dt,), None, "poisson_solve_noalloc p")
    precision = VF_FP64 if dt == "float64" else VF_FP32_MIXED
    if _noalloc_sizes_accepted(nx, ny, nz, precision):   # sizes the call refuses never reach the arrays
        for x, what in ((f, "f"), (p, "p")):
            if x.numel() != nx * ny * nz:
                raise ValueError(f"poisson_solve_noalloc {what}: expected {nx * ny * nz} elements, got {x.numel()}")
    rc = lib().vf_poisson_solve_noalloc(nx, ny, nz, lx, ly, lz, precision, C.c_void_p(f.data_ptr()),
                                        C.c_void_p(p.data_ptr()), C.c_void_p(stream) if stream else None)
    if rc != VF_OK:
        raise VentflowError(rc, "vf_poisson_solve_noalloc")


# -- host-side ventilation metrics
def ach_log_slope(t_seconds, c_mean):
    t = np.ascontiguousarray(t_seconds, dtype=np.float64)
    c = np.ascontiguousarray(c_mean, dtype=np.float64)
    out = C.c_double()
    rc = lib().vf_ach_log_slope(_dptr(t), _dptr(c), t.size, C.byref(out))
    if rc != VF_OK:
        raise VentflowError(rc, "vf_ach_log_slope")
    return out.value


def ach_fit3(t_seconds, c_mean):
    t = np.ascontiguousarray(t_seconds, dtype=np.float64)
    c = np.ascontiguousarray(c_mean, dtype=np.float64)
    a, c0, c1 = C.c_double(), C.c_double(), C.c_double()
    rc = lib().vf_ach_fit3(_dptr(t), _dptr(c), t.size, C.byref(a), C.byref(c0), C.byref(c1))
    if rc != VF_OK:
        raise VentflowError(rc, "vf_ach_fit3")
    return a.value, c0.value, c1.value


def wells_riley(c0, breathing_m3_h, ach_per_hour, t_hours):
    q, p = C.c_double(), C.c_double()
    rc = lib().vf_wells_riley(float(c0), float(breathing_m3_h), float(ach_per_hour), float(t_hours), C.byref(q),
                              C.byref(p))
    if rc != VF_OK:
        raise VentflowError(rc, "vf_wells_riley")
    return q.value, p.value


def room_grid(room, precision="fp32", filter=True, n_pressure_iters=4, nu=1.6e-5, dt=None, **kw):
    """A Grid set up for a ``rooms.Room``: mask, forcing region (u_set = (U_in, 0, 0), c_set = 0), room region
    and the stale-air initial scalar."""
    g = Grid(room.nx, room.ny, room.nz, room.lx, room.ly, room.lz, nu=nu, dt=room.dt if dt is None else dt,
             filter=filter, n_pressure_iters=n_pressure_iters, precision=precision, **kw)
    g.set_mask(room.beta)
    g.set_inflow(room.S, (room.u_in, 0.0, 0.0), 0.0)
    g.set_region(room.room)
    g.set_field("c", room.initial_c())
    return g
