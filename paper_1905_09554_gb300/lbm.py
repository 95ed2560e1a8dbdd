"""Thin ctypes binding of the C ABI in include/lbm_sc.h.

Argument marshalling only: every step of the method runs in the CUDA library
``liblbm_sc.so``.  If the library is missing or cannot be loaded, every entry
point raises; there is no CPU fallback.

The module-level functions carry the C names (``lbm_create``, ``lbm_step``
...) and return the raw ``lbm_status``; :class:`Lattice` wraps a context,
raises :class:`LbmError` on failure, and can keep the two population copies
in PyTorch device memory on the current PyTorch stream.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblbm_sc.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "lbm_sc.h")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EIO, LBM_EUNSUPPORTED = range(8)
STATUS_NAMES = ["LBM_OK", "LBM_EINVAL", "LBM_ENOMEM", "LBM_ECUDA", "LBM_ENONFINITE",
                "LBM_ETIMEOUT", "LBM_EIO", "LBM_EUNSUPPORTED"]
LBM_D3Q19 = 0
LBM_SRT_SHIFT, LBM_MRT_GUO = 0, 1
LBM_PSI_EXP = 0
LBM_F64, LBM_F32, LBM_F16_DEV, LBM_BF16_DEV, LBM_F16_LOCAL, LBM_BF16_LOCAL = 0, 1, 2, 3, 4, 5
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16_DEV, "bf16": LBM_BF16_DEV,
           "f16l": LBM_F16_LOCAL, "bf16l": LBM_BF16_LOCAL}
STORAGE_BYTES = {LBM_F64: 8, LBM_F32: 4, LBM_F16_DEV: 2, LBM_BF16_DEV: 2, LBM_F16_LOCAL: 2, LBM_BF16_LOCAL: 2}
COLLISION = {"srt": LBM_SRT_SHIFT, "mrt": LBM_MRT_GUO}


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("G", ctypes.c_double),
        ("collision", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("has_rates", ctypes.c_int),
        ("s", ctypes.c_double * 19),
        ("psi", ctypes.c_int),
        ("rho0", ctypes.c_double),
        ("storage", ctypes.c_int),
        ("rho_ref", ctypes.c_double),
        ("dev_scale", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("f_a", ctypes.c_void_p), ("f_b", ctypes.c_void_p),
        ("zchunk", ctypes.c_int),
        ("tile_y", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("test_stall", ctypes.c_int),
        ("G2", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "lbm_params_default": (None, [ctypes.POINTER(lbm_params)]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.POINTER(_P)]),
    "lbm_destroy": (None, [_P]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_velocities": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), _D]),
    "lbm_init_ligament": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lbm_set_density": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "lbm_set_populations": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "lbm_get_populations": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "lbm_step": (ctypes.c_int, [_P, ctypes.c_long]),
    "lbm_time": (ctypes.c_long, [_P]),
    "lbm_current_copy": (ctypes.c_int, [_P]),
    "lbm_moments": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "lbm_diag": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D]),
    "lbm_set_stream": (ctypes.c_int, [_P, _P]),
    "lbm_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lbm_checkpoint_info": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
    "lbm_device_bytes": (ctypes.c_longlong, [_P]),
    "lbm_params_sizeof": (ctypes.c_longlong, []),
    "lbm_kernel_config": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_set_kernel_config": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_tune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), _D]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(_P)]),
    "lbm_batch_destroy": (None, [_P]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_batch_box": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "lbm_batch_step": (ctypes.c_int, [_P, ctypes.c_long]),
    "lbm_batch_tune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      _D]),
    "lbm_batch_config": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_adjoint_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_long, ctypes.c_int]),
    "lbm_adjoint_backward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _D, _D]),
    "lbm_diag_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        _P, _P, _P, _P, ctypes.c_int, _P]),
}

_lib = None


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/lbm_sc.h."""
    text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M)))


def load(path: str | None = None):
    """Load liblbm_sc.so (building it first if it is absent and nvcc exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        from . import build as _build
        p = _build.build()
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.lbm_params_sizeof() != ctypes.sizeof(lbm_params):
        raise RuntimeError("lbm_params layout mismatch between binding and library")
    if path is None:
        _lib = lib
    return lib


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


# ------------------------------------------------------------ C-named calls
def lbm_params_default() -> lbm_params:
    p = lbm_params()
    load().lbm_params_default(ctypes.byref(p))
    return p


def lbm_create(p: lbm_params):
    ctx = _P()
    st = load().lbm_create(ctypes.byref(p), ctypes.byref(ctx))
    return st, ctx


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_last_error(ctx=None) -> str:
    return (load().lbm_last_error(ctx) or b"").decode()


def lbm_velocities():
    c = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    load().lbm_velocities(c, w)
    return np.array(c[:], dtype=np.int64).reshape(19, 3), np.array(w[:])


def lbm_init_ligament(ctx, R0, eps, n_waves, width, rho_l, rho_v):
    return load().lbm_init_ligament(ctx, R0, eps, n_waves, width, rho_l, rho_v)


def lbm_set_density(ctx, ptr, on_device):
    return load().lbm_set_density(ctx, ptr, on_device)


def lbm_set_populations(ctx, ptr, on_device):
    return load().lbm_set_populations(ctx, ptr, on_device)


def lbm_get_populations(ctx, ptr, on_device):
    return load().lbm_get_populations(ctx, ptr, on_device)


def lbm_step(ctx, n):
    return load().lbm_step(ctx, n)


def lbm_time(ctx):
    return load().lbm_time(ctx)


def lbm_current_copy(ctx):
    return load().lbm_current_copy(ctx)


def lbm_moments(ctx, rho, ux, uy, uz, on_device):
    return load().lbm_moments(ctx, rho, ux, uy, uz, on_device)


def lbm_diag(ctx, rho_l, rho_v, mass, mom, area_z, maxrho_z):
    return load().lbm_diag(ctx, rho_l, rho_v, mass, mom, area_z, maxrho_z)


def lbm_set_stream(ctx, stream):
    return load().lbm_set_stream(ctx, stream)


def lbm_save(ctx, path):
    return load().lbm_save(ctx, os.fsencode(path))


def lbm_load(ctx, path):
    return load().lbm_load(ctx, os.fsencode(path))


def lbm_checkpoint_info(path, verify=True):
    """(status, dict(dims=(nx, ny, nz), storage, collision, t, G, tau)) of a
    checkpoint file, read on the host alone."""
    dims = (ctypes.c_int * 3)()
    st_, co, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
    G, tau = ctypes.c_double(), ctypes.c_double()
    st = load().lbm_checkpoint_info(os.fsencode(path), 1 if verify else 0, dims, ctypes.byref(st_),
                                    ctypes.byref(co), ctypes.byref(t), ctypes.byref(G), ctypes.byref(tau))
    return st, dict(dims=tuple(dims), storage=st_.value, collision=co.value, t=t.value, G=G.value, tau=tau.value)


def checkpoint_info(path, verify=True):
    """Header of a checkpoint (lbm_checkpoint_info); raises LbmError on a bad file."""
    st, info = lbm_checkpoint_info(path, verify)
    if st != LBM_OK:
        raise LbmError(st, lbm_last_error(None))
    return info


def lbm_device_bytes(ctx):
    return load().lbm_device_bytes(ctx)


def lbm_adjoint_forward(ctx, rho0, on_device, n, every):
    return load().lbm_adjoint_forward(ctx, rho0, on_device, n, every)


def lbm_adjoint_backward(ctx, dJdrho, in_on_device, dJdrho0, out_on_device, dJdG, dJdtau):
    return load().lbm_adjoint_backward(ctx, dJdrho, in_on_device, dJdrho0, out_on_device, dJdG, dJdtau)


def lbm_batch_create(p: lbm_params, dims):
    arr = (ctypes.c_int * (3 * len(dims)))(*[int(v) for d in dims for v in d])
    b = _P()
    st = load().lbm_batch_create(ctypes.byref(p), len(dims), arr, ctypes.byref(b))
    return st, b


def lbm_batch_destroy(b):
    load().lbm_batch_destroy(b)


def lbm_batch_last_error(b=None) -> str:
    return (load().lbm_batch_last_error(b) or b"").decode()


def lbm_batch_box(b, i):
    v = _P()
    st = load().lbm_batch_box(b, i, ctypes.byref(v))
    return st, v


def lbm_batch_step(b, n):
    return load().lbm_batch_step(b, n)


def lbm_batch_tune(b, trial_steps):
    ty, zc, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = load().lbm_batch_tune(b, trial_steps, ctypes.byref(ty), ctypes.byref(zc), ctypes.byref(ms))
    return st, dict(tile_y=ty.value, zchunk=zc.value, ms_per_step=ms.value)


def lbm_batch_config(b):
    v = [ctypes.c_int() for _ in range(3)]
    cells = ctypes.c_longlong()
    st = load().lbm_batch_config(b, *[ctypes.byref(x) for x in v], ctypes.byref(cells))
    return st, dict(tile_y=v[0].value, zchunk=v[1].value, grid=v[2].value, cells=cells.value)


def lbm_diag_noalloc(f, storage, nx, ny, nz, rho_ref, dev_scale, rho_l, rho_v, mass, mom, area_z,
                     maxrho_z, on_device, stream):
    """Allocation-free diagnostics on a caller-owned population array (see
    include/lbm_sc.h); pointers are passed through unchanged."""
    return load().lbm_diag_noalloc(f, storage, nx, ny, nz, rho_ref, dev_scale, rho_l, rho_v, mass, mom,
                                   area_z, maxrho_z, on_device, stream)


def lbm_kernel_config(ctx):
    v = [ctypes.c_int() for _ in range(4)]
    st = load().lbm_kernel_config(ctx, *[ctypes.byref(x) for x in v])
    return st, dict(zip(("kernel", "tile_y", "zchunk", "grid"), (x.value for x in v)))


# ------------------------------------------------------------ object wrapper
def lbm_set_kernel_config(ctx, kernel, tile_y, zchunk):
    return load().lbm_set_kernel_config(ctx, int(kernel), int(tile_y), int(zchunk))


def lbm_tune(ctx, trial_steps):
    k, t, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    st = load().lbm_tune(ctx, int(trial_steps), ctypes.byref(k), ctypes.byref(t), ctypes.byref(z), ctypes.byref(ms))
    return st, {"kernel": k.value, "tile_y": t.value, "zchunk": z.value, "ms_per_step": ms.value}


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _host_array(a, numel, what):
    """float64 C-contiguous copy (or view) of a host array of numel values."""
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.size != numel:
        raise ValueError(f"{what}: expected {numel} values, got {arr.size}")
    return arr


def _device_tensor(t, numel, what):
    """Check a CUDA float64 contiguous tensor of numel values (the library
    reads or writes it in place, so no conversion is made)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a numpy array or a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{what}: need a contiguous float64 CUDA tensor of {numel} values "
                         f"(got {t.dtype}, contiguous={t.is_contiguous()}, {t.numel()} values)")
    return t.data_ptr()


def _params(G=-5.5, tau=1.0, collision="srt", rates=None, storage="f32", rho0=1.0, rho_ref=1.0,
            dev_scale=1.0, zchunk=0, tile_y=0, kernel=0):
    if collision not in COLLISION:
        raise ValueError(f"collision must be one of {sorted(COLLISION)}, got {collision!r}")
    if storage not in STORAGE:
        raise ValueError(f"storage must be one of {sorted(STORAGE)}, got {storage!r}")
    p = lbm_params_default()
    p.G, p.tau, p.rho0 = float(G), float(tau), float(rho0)
    p.collision = COLLISION[collision]
    if rates is not None:
        rates = [float(v) for v in rates]
        if len(rates) != 19:
            raise ValueError(f"rates: expected 19 MRT rates, got {len(rates)}")
        p.has_rates = 1
        for k, v in enumerate(rates):
            p.s[k] = v
    p.storage = STORAGE[storage]
    p.rho_ref, p.dev_scale = float(rho_ref), float(dev_scale)
    p.zchunk, p.tile_y, p.kernel = int(zchunk), int(tile_y), int(kernel)
    return p


class Lattice:
    """One periodic D3Q19 Shan-Chen lattice on the current CUDA device.

    collision: 'srt' (shifted velocity) or 'mrt' (Guo forcing); rates: None
    (the paper's rule), or 19 MRT rates in moment order.  storage: 'f64',
    'f32', 'f16' or 'bf16' (deviations from a global rho_ref), 'f16l' or
    'bf16l' (deviations from a per-cell reference density).  With torch_buffers=True the two population
    copies are torch.cuda tensors owned by this object and all work runs on
    torch's current stream.
    """

    def __init__(self, nx, ny, nz, G=-5.5, tau=1.0, collision="srt", rates=None,
                 storage="f32", rho0=1.0, rho_ref=1.0, dev_scale=1.0,
                 torch_buffers=True, stream=None, zchunk=0, tile_y=0, kernel=0, test_stall=0, G2=0.0):
        lib = load()
        p = _params(G, tau, collision, rates, storage, rho0, rho_ref, dev_scale, zchunk, tile_y, kernel)
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.test_stall = int(test_stall)
        p.G2 = float(G2)
        self.shape = (int(nz), int(ny), int(nx))
        self.n = int(nx) * int(ny) * int(nz)
        self.storage = storage
        self._bufs = None
        self._torch_stream = None
        if stream is not None:
            p.stream = int(stream)
        if torch_buffers:
            import torch
            if not torch.cuda.is_available():
                raise LbmError(LBM_ECUDA, "no CUDA device visible to torch")
            nbytes = 19 * self.n * STORAGE_BYTES[p.storage]
            self._bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
            p.f_a, p.f_b = self._bufs[0].data_ptr(), self._bufs[1].data_ptr()
            if stream is None:
                self._torch_stream = torch.cuda.current_stream()
                p.stream = self._torch_stream.cuda_stream
        self.params = p
        st, ctx = lbm_create(p)
        if st != LBM_OK:
            raise LbmError(st, lbm_last_error(None))
        self.ctx = ctx
        self._lib = lib

    # -- helpers
    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, lbm_last_error(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None
        self._bufs = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def time(self):
        return lbm_time(self.ctx)

    def stored_populations(self):
        """The torch uint8 buffer that holds the current state exactly as
        stored (19 * nx * ny * nz elements of the storage type, library
        velocity order); only with torch_buffers=True."""
        if self._bufs is None:
            raise LbmError(LBM_EINVAL, "stored_populations: the population copies are not torch buffers")
        return self._bufs[lbm_current_copy(self.ctx)]

    # -- state
    def init_ligament(self, R0, eps, rho_l, rho_v, width=2.0, n_waves=1):
        self._check(lbm_init_ligament(self.ctx, R0, eps, n_waves, width, rho_l, rho_v))

    def set_density(self, rho):
        """rho: numpy float64 (nz, ny, nx) or a contiguous float64 CUDA tensor."""
        if isinstance(rho, np.ndarray):
            a = _host_array(rho, self.n, "set_density")
            self._check(lbm_set_density(self.ctx, _host_ptr(a), 0))
        else:
            self._check(lbm_set_density(self.ctx, _device_tensor(rho, self.n, "set_density"), 1))

    def set_populations(self, f):
        if isinstance(f, np.ndarray):
            a = _host_array(f, 19 * self.n, "set_populations")
            self._check(lbm_set_populations(self.ctx, _host_ptr(a), 0))
        else:
            self._check(lbm_set_populations(self.ctx, _device_tensor(f, 19 * self.n, "set_populations"), 1))

    def get_populations(self, out=None):
        """float64 populations (19, nz, ny, nx), library velocity order; into
        a CUDA tensor ``out`` if given, else a new numpy array."""
        if out is not None:
            self._check(lbm_get_populations(self.ctx, _device_tensor(out, 19 * self.n, "get_populations"), 1))
            return out
        a = np.empty((19,) + self.shape)
        self._check(lbm_get_populations(self.ctx, _host_ptr(a), 0))
        return a

    def step(self, n=1):
        self._check(lbm_step(self.ctx, int(n)))

    def moments(self):
        """(rho, u) as numpy float64; u = (ux, uy, uz) barycentric."""
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self._check(lbm_moments(self.ctx, _host_ptr(rho), _host_ptr(u[0]), _host_ptr(u[1]),
                                _host_ptr(u[2]), 0))
        return rho, u

    def density(self):
        """rho alone as numpy float64 (nz, ny, nx): a quarter of moments()'s
        host memory and transfer."""
        rho = np.empty(self.shape)
        self._check(lbm_moments(self.ctx, _host_ptr(rho), None, None, None, 0))
        return rho

    def moments_device(self, rho, ux=None, uy=None, uz=None):
        """rho and u_b into CUDA float64 tensors of nx*ny*nz values (any may be
        None)."""
        def ptr(t):
            return None if t is None else _device_tensor(t, self.n, "moments_device")

        self._check(lbm_moments(self.ctx, ptr(rho), ptr(ux), ptr(uy), ptr(uz), 1))

    def diag(self, rho_l, rho_v, raise_nonfinite=True):
        """dict(mass, mom (3,), area_z (nz,), maxrho_z (nz,), status)."""
        nz = self.shape[0]
        mass = ctypes.c_double()
        mom = (ctypes.c_double * 3)()
        area = np.empty(nz)
        mx = np.empty(nz)
        st = lbm_diag(self.ctx, rho_l, rho_v, ctypes.byref(mass), mom,
                      area.ctypes.data_as(_D), mx.ctypes.data_as(_D))
        if st != LBM_OK and (raise_nonfinite or st != LBM_ENONFINITE):
            self._check(st)
        return dict(mass=mass.value, mom=np.array(mom[:]), area_z=area, maxrho_z=mx, status=st)

    def device_bytes(self):
        return lbm_device_bytes(self.ctx)

    def adjoint_forward(self, rho0, n, every):
        """Run n steps from rest with density rho0 keeping checkpoints."""
        if isinstance(rho0, np.ndarray):
            a = _host_array(rho0, self.n, "adjoint_forward")
            self._check(lbm_adjoint_forward(self.ctx, _host_ptr(a), 0, int(n), int(every)))
        else:
            self._check(lbm_adjoint_forward(self.ctx, _device_tensor(rho0, self.n, "adjoint_forward"), 1, int(n),
                                            int(every)))

    def adjoint_backward(self, dJdrho, out=None):
        """Returns (dJ/drho0, dJ/dG, dJ/dtau); dJdrho and out may be numpy
        arrays or CUDA float64 tensors."""
        dG, dT = ctypes.c_double(), ctypes.c_double()
        if isinstance(dJdrho, np.ndarray):
            g = _host_array(dJdrho, self.n, "adjoint_backward")
            gp, gdev = _host_ptr(g), 0
        else:
            gp, gdev = _device_tensor(dJdrho, self.n, "adjoint_backward"), 1
        if out is None:
            res = np.empty(self.shape)
            op, odev = _host_ptr(res), 0
        else:
            res, op, odev = out, _device_tensor(out, self.n, "adjoint_backward out"), 1
        self._check(lbm_adjoint_backward(self.ctx, gp, gdev, op, odev, ctypes.byref(dG), ctypes.byref(dT)))
        return res, dG.value, dT.value

    def save(self, path):
        """Checkpoint the current state to `path` (lbm_save)."""
        self._check(lbm_save(self.ctx, path))

    def load(self, path):
        """Restore a state written by save() (lbm_load)."""
        self._check(lbm_load(self.ctx, path))

    def kernel_config(self):
        st, cfg = lbm_kernel_config(self.ctx)
        self._check(st)
        return cfg

    def set_kernel_config(self, kernel=0, tile_y=0, zchunk=0):
        self._check(lbm_set_kernel_config(self.ctx, kernel, tile_y, zchunk))

    def tune(self, trial_steps=3, cache=None):
        """Pick the step's launch shape (kernel variant, tile height, z chunk)
        by timing the candidates on this lattice (lbm_tune); tune before
        setting the initial state, since the trial steps advance it.  With
        `cache` (a JSON file path) a pick stored for the same box, parameters
        and GPU model is applied without timing, and a new pick is stored.
        Returns the pick (kernel, tile_y, zchunk, ms_per_step, cached)."""
        key = None
        if cache is not None:
            p = self.params
            phys = {"storage": self.storage, "collision": int(p.collision), "G": p.G, "G2": p.G2, "tau": p.tau,
                    "rates": [p.s[k] for k in range(19)] if p.has_rates else None}
            key = "lattice:" + _tune_key([self.shape[::-1]], phys)
            hit = _read_tune_cache(cache).get(key)
            if hit:
                self.set_kernel_config(hit["kernel"], hit["tile_y"], hit["zchunk"])
                return dict(hit, cached=True)
        st, pick = lbm_tune(self.ctx, trial_steps)
        self._check(st)
        if key is not None:
            data = _read_tune_cache(cache)
            data[key] = pick
            _write_tune_cache(cache, data)
        return dict(pick, cached=False)


class _BoxView(Lattice):
    """Lattice-like access to one box of a Batch (no buffers of its own)."""

    def __init__(self, batch, i, ctx, shape):
        self.ctx = ctx
        self.shape = shape
        self.n = shape[0] * shape[1] * shape[2]
        self._bufs = None
        self._batch = batch
        self.index = i

    def close(self):
        self.ctx = None  # owned by the batch

    def step(self, n=1):
        raise LbmError(LBM_EINVAL, "boxes of a batch are stepped together with Batch.step")


def _tune_key(dims, kw):
    """Cache key of a batch's launch-shape pick: the boxes, the physics
    keywords and the GPU model."""
    import hashlib
    import json
    try:
        import torch
        gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    except Exception:
        gpu = "none"
    blob = json.dumps({"dims": [[int(v) for v in d] for d in dims], "gpu": gpu,
                       "params": {k: kw[k] for k in sorted(kw) if k not in ("tile_y", "zchunk")}},
                      sort_keys=True, default=str)
    return hashlib.sha256(blob.encode()).hexdigest()[:20]


def _read_tune_cache(path):
    import json
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _write_tune_cache(path, data):
    import json
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Batch:
    """Independent periodic boxes (dims: list of (nx, ny, nz)) advanced
    together; the physics keywords are those of Lattice (FP32/FP64 only).

    tune_cache: path of a JSON file of launch-shape picks.  When given (and
    neither tile_y nor zchunk is), a pick stored for the same boxes, physics
    and GPU model is used; otherwise the batch is autotuned once at creation
    (lbm_batch_tune, before any state is set) and its pick stored."""

    def __init__(self, dims, stream=None, tune_cache=None, trial_steps=3, **kw):
        load()
        key = cached = None
        if tune_cache is not None and "tile_y" not in kw and "zchunk" not in kw:
            key = _tune_key(dims, kw)
            cached = _read_tune_cache(tune_cache).get(key)
            if cached:
                kw = dict(kw, tile_y=int(cached["tile_y"]), zchunk=int(cached["zchunk"]))
        p = _params(**kw)
        if stream is not None:
            p.stream = int(stream)
        else:
            import torch
            if torch.cuda.is_available():
                s = torch.cuda.current_stream().cuda_stream
                p.stream = s if s else None
        st, b = lbm_batch_create(p, dims)
        if st != LBM_OK:
            raise LbmError(st, lbm_batch_last_error(None))
        self.b = b
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.boxes = []
        for i, (nx, ny, nz) in enumerate(self.dims):
            st, v = lbm_batch_box(b, i)
            self._check(st)
            self.boxes.append(_BoxView(self, i, v, (nz, ny, nx)))
        if key is not None and not cached:
            best = self.tune(trial_steps)
            data = _read_tune_cache(tune_cache)
            data[key] = {"tile_y": best["tile_y"], "zchunk": best["zchunk"], "ms_per_step": best["ms_per_step"]}
            _write_tune_cache(tune_cache, data)

    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, lbm_batch_last_error(self.b))

    def step(self, n=1):
        self._check(lbm_batch_step(self.b, int(n)))

    def tune(self, trial_steps=3):
        st, r = lbm_batch_tune(self.b, int(trial_steps))
        self._check(st)
        return r

    def config(self):
        st, r = lbm_batch_config(self.b)
        self._check(st)
        return r

    def close(self):
        if getattr(self, "b", None):
            for v in self.boxes:
                v.ctx = None
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

