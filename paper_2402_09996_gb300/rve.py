"""ctypes binding of librve.so (include/rve.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module converts
numpy arrays / torch tensors to pointers, passes torch's current CUDA stream and,
optionally, torch's caching allocator, and turns status codes into exceptions.
If librve.so cannot be loaded or no CUDA device is usable, calls raise: there is
no CPU path.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "librve.so"

FP64, FP32 = 0, 1
GREEN_WILLOT, GREEN_MS = 0, 1
FIELD_STRESS, FIELD_STRAIN, FIELD_EPS_P, FIELD_V, FIELD_ALPHA, FIELD_VM, FIELD_F = range(7)
FIELD_COMPONENTS = {FIELD_STRESS: 6, FIELD_STRAIN: 6, FIELD_EPS_P: 6, FIELD_V: 16, FIELD_ALPHA: 12, FIELD_VM: 1,
                    FIELD_F: 4}
DTYPE_F64, DTYPE_F32 = 0, 1
KERNELS = ["xpass", "yfwd", "zgreen", "yinv", "commit", "shift", "idle"]
STATUS = {
    0: "RVE_OK",
    1: "RVE_ERR_INVALID_ARG",
    2: "RVE_ERR_CUDA",
    3: "RVE_ERR_OOM",
    4: "RVE_ERR_NOT_CONVERGED",
    5: "RVE_ERR_NAN",
    6: "RVE_ERR_STATE",
    7: "RVE_ERR_UNSUPPORTED",
}
STATUS_CODES = {name: code for code, name in STATUS.items()}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("green", C.c_int),
        ("n_sub", C.c_int),
        ("max_iter", C.c_int),
        ("fixed_iters", C.c_int),
        ("tol", C.c_double),
        ("stream", C.c_void_p),
        ("device", C.c_int),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", C.c_void_p),
        ("timing", C.c_int),
        ("graphs", C.c_int),
        ("autotune", C.c_int),
        ("y_tile", C.c_int),
        ("z_tile", C.c_int),
        ("batch_group", C.c_int),
        ("c0_lambda", C.c_double),
        ("c0_mu", C.c_double),
    ]


MATERIAL_FIELDS = [
    "C11", "C12", "C13", "C33", "C44", "C66", "r0_ord", "r0_sup", "r0_twin", "K", "n", "Kt", "nt",
    "Q_s", "Q_b", "b_s", "b_b", "h_diag", "h_off", "c", "d", "Kc", "fm", "eta",
]


class Material(C.Structure):
    _fields_ = [(f, C.c_double) for f in MATERIAL_FIELDS]

    def as_dict(self):
        return {f: getattr(self, f) for f in MATERIAL_FIELDS}


class Effective(C.Structure):
    _fields_ = [
        ("increment", C.c_int),
        ("iterations", C.c_int),
        ("time", C.c_double),
        ("E", C.c_double * 6),
        ("S", C.c_double * 6),
        ("S_eq_of_mean", C.c_double),
        ("mean_S_eq", C.c_double),
        ("mean_f", C.c_double),
        ("mean_v", C.c_double),
        ("residual", C.c_double),
        ("stress_residual", C.c_double),
    ]

    def as_dict(self):
        return {
            "increment": self.increment,
            "iterations": self.iterations,
            "time": self.time,
            "E": np.array(self.E[:]),
            "S": np.array(self.S[:]),
            "S_eq_of_mean": self.S_eq_of_mean,
            "mean_S_eq": self.mean_S_eq,
            "mean_f": self.mean_f,
            "mean_v": self.mean_v,
            "residual": self.residual,
            "stress_residual": self.stress_residual,
        }


class RVEError(RuntimeError):
    def __init__(self, status: int, message: str, index: int = -1):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.index = index  # failing solver of a batch call, else -1


_lib = None

EXPORTED = [
    "rve_options_default", "rve_material_default", "rve_create", "rve_set_material",
    "rve_set_mixed_load", "rve_step", "rve_get_effective", "rve_get_fields", "rve_save_state",
    "rve_load_state", "rve_last_error", "rve_destroy", "rve_material_point", "rve_fft_r2c",
    "rve_fft_c2r", "rve_label_voronoi", "rve_kernel_times", "rve_get_residuals", "rve_label_voronoi_noalloc",
    "rve_step_batch", "rve_material_point_vjp", "rve_adjoint_increment", "rve_alu_probe", "rve_batch_grouped",
    "rve_get_fields_as",
]
NOALLOC_MAX_PARENTS = 4096  # RVE_NOALLOC_MAX_PARENTS of include/rve.h


def load_library(path: str | os.PathLike | None = None):
    """Load librve.so (raises OSError when missing: build it with build_lib.build())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise OSError(f"{p} not found; build it with paper_2402_09996_gb300.build_lib.build()")
    lib = C.CDLL(str(p))
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    lib.rve_options_default.argtypes = [C.POINTER(Options)]
    lib.rve_material_default.argtypes = [C.POINTER(Material)]
    lib.rve_create.argtypes = [C.POINTER(vp), i, i, i, vp, i, i, vp, C.POINTER(Options)]
    lib.rve_set_material.argtypes = [vp, C.POINTER(Material)]
    lib.rve_set_mixed_load.argtypes = [vp, vp, vp, vp, d]
    lib.rve_step.argtypes = [vp, i, C.POINTER(C.c_longlong)]
    lib.rve_get_effective.argtypes = [vp, C.POINTER(Effective), C.POINTER(Effective), i, C.POINTER(i)]
    lib.rve_get_fields.argtypes = [vp, i, vp, sz, i]
    lib.rve_get_fields_as.argtypes = [vp, i, i, vp, sz, i]
    lib.rve_save_state.argtypes = [vp, vp, C.POINTER(sz)]
    lib.rve_load_state.argtypes = [vp, vp, sz]
    lib.rve_last_error.argtypes = [vp]
    lib.rve_last_error.restype = C.c_char_p
    lib.rve_destroy.argtypes = [vp]
    lib.rve_destroy.restype = None
    lib.rve_material_point.argtypes = [i, C.POINTER(Material), C.c_longlong, vp, vp, vp, vp, vp, d, i, vp]
    lib.rve_fft_r2c.argtypes = [i, i, i, i, i, vp, vp, vp]
    lib.rve_fft_c2r.argtypes = [i, i, i, i, i, vp, vp, vp]
    lib.rve_label_voronoi.argtypes = [i, i, i, i, vp, vp, vp, vp, i, vp]
    lib.rve_kernel_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), i]
    lib.rve_get_residuals.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), i, C.POINTER(i)]
    lib.rve_label_voronoi_noalloc.argtypes = [i, i, i, i, vp, vp, vp, vp, vp]
    lib.rve_step_batch.argtypes = [C.POINTER(vp), i, i, C.POINTER(C.c_longlong), C.POINTER(i)]
    lib.rve_material_point_vjp.argtypes = [i, C.POINTER(Material), C.c_longlong, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                           vp, d, i, vp]
    lib.rve_adjoint_increment.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_double), d, vp, vp, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    lib.rve_alu_probe.argtypes = [i, i, i, vp, vp, C.POINTER(C.c_double)]
    lib.rve_batch_grouped.argtypes = [C.POINTER(vp), i, C.POINTER(i)]
    for name in EXPORTED:
        getattr(lib, name).restype = C.c_int
    lib.rve_options_default.restype = None
    lib.rve_material_default.restype = None
    lib.rve_last_error.restype = C.c_char_p
    lib.rve_destroy.restype = None
    _lib = lib
    return lib


def _check(status: int, handle=None):
    if status != 0:
        msg = _lib.rve_last_error(handle).decode(errors="replace")
        raise RVEError(status, msg)


def default_material() -> Material:
    lib = load_library()
    m = Material()
    lib.rve_material_default(C.byref(m))
    return m


def default_options() -> Options:
    lib = load_library()
    o = Options()
    lib.rve_options_default(C.byref(o))
    return o


def _torch_stream():
    import torch

    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class _TorchAllocator:
    """Device allocations through torch's caching allocator on the current stream."""

    def __init__(self, device: int):
        import torch

        self.torch = torch
        self.device = device
        self.stream = torch.cuda.current_stream(device)

        def _alloc(nbytes, _ctx):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # noqa: BLE001 - reported to the library as a NULL pointer
                return None

        def _free(ptr, _ctx):
            if ptr:
                self.torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def _ptr(a) -> C.c_void_p:
    """Device pointer of a torch tensor or host pointer of a C-contiguous numpy array."""
    if a is None:
        return C.c_void_p(None)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


class RVE:
    """One periodic voxel RVE solved on the GPU (wraps an rve_t handle).

    grain_id: (nz, ny, nx) integer labels (x fastest), numpy (host) or torch CUDA tensor;
    euler: (n_grains, 3) Bunge angles [rad].
    """

    def __init__(self, grain_id, euler, precision=FP64, green=GREEN_WILLOT, n_sub=0, tol=1e-6, max_iter=1000,
                 fixed_iters=0, device=0, use_torch=True, timing=False, graphs=True, autotune=True, y_tile=0,
                 z_tile=0, batch_group=False, c0=None):
        self.lib = load_library()
        euler = np.ascontiguousarray(np.asarray(euler, dtype=np.float64))
        shape = tuple(grain_id.shape)
        if len(shape) != 3:
            raise ValueError("grain_id must have shape (nz, ny, nx)")
        self.shape = shape
        self.nvox = int(np.prod(shape))
        opt = default_options()
        opt.precision, opt.green, opt.n_sub = precision, green, n_sub
        opt.tol, opt.max_iter, opt.fixed_iters, opt.device = tol, max_iter, fixed_iters, device
        opt.timing = 1 if timing else 0
        opt.graphs = 1 if graphs else 0
        opt.autotune = 1 if autotune else 0
        opt.y_tile, opt.z_tile = int(y_tile), int(z_tile)
        opt.batch_group = 1 if batch_group else 0
        if c0 is not None:  # (lambda0, mu0) of the reference medium [MPa]
            opt.c0_lambda, opt.c0_mu = float(c0[0]), float(c0[1])
        self._allocator = None
        on_dev = 0
        if use_torch:
            import torch

            with torch.cuda.device(device):
                opt.stream = _torch_stream()
                self._allocator = _TorchAllocator(device)
            opt.alloc, opt.free = self._allocator.alloc, self._allocator.free
        if hasattr(grain_id, "data_ptr"):
            gid = grain_id.contiguous()
            if str(gid.dtype) not in ("torch.int32", "torch.uint32"):
                raise TypeError("device grain_id must be int32/uint32")
            on_dev = 1 if gid.is_cuda else 0
            if not gid.is_cuda:
                gid = gid.numpy().astype(np.uint32)
        else:
            gid = np.ascontiguousarray(np.asarray(grain_id).astype(np.uint32))
        self._gid_keepalive = gid
        h = C.c_void_p()
        nz, ny, nx = shape
        st = self.lib.rve_create(C.byref(h), nx, ny, nz, _ptr(gid), on_dev, euler.shape[0], _ptr(euler), C.byref(opt))
        _check(st, None)
        self.h = h

    # ---- configuration ------------------------------------------------------
    def set_material(self, **kw):
        m = default_material()
        for k, v in kw.items():
            if k not in MATERIAL_FIELDS:
                raise KeyError(k)
            setattr(m, k, float(v))
        _check(self.lib.rve_set_material(self.h, C.byref(m)), self.h)

    def set_mixed_load(self, Edot=(0, 0, 1e-3, 0, 0, 0), strain_ctrl=(0, 0, 1, 0, 0, 0), Sigma=(0,) * 6, dt=1.0):
        e = np.ascontiguousarray(Edot, dtype=np.float64)
        c = np.ascontiguousarray(strain_ctrl, dtype=np.uint8)
        s = np.ascontiguousarray(Sigma, dtype=np.float64)
        _check(self.lib.rve_set_mixed_load(self.h, _ptr(e), _ptr(c), _ptr(s), float(dt)), self.h)

    # ---- solve ----------------------------------------------------------------
    def step(self, n_increments=1) -> int:
        it = C.c_longlong(0)
        _check(self.lib.rve_step(self.h, int(n_increments), C.byref(it)), self.h)
        return int(it.value)

    def effective(self) -> dict:
        e = Effective()
        _check(self.lib.rve_get_effective(self.h, C.byref(e), None, 0, None), self.h)
        return e.as_dict()

    def history(self) -> list:
        n = C.c_int(0)
        _check(self.lib.rve_get_effective(self.h, None, None, 0, C.byref(n)), self.h)
        arr = (Effective * max(1, n.value))()
        _check(self.lib.rve_get_effective(self.h, None, arr, n.value, None), self.h)
        return [arr[i].as_dict() for i in range(n.value)]

    def field(self, which: int, out=None, dtype=np.float64):
        """Committed field (components, nz, ny, nx) as float64 or float32 (`dtype`); `out`
        may be a CUDA tensor of that type."""
        comps = FIELD_COMPONENTS[which]
        single = np.dtype(dtype) == np.float32 if out is None else str(out.dtype) in ("torch.float32", "float32")
        if out is None:
            out = np.empty((comps,) + self.shape, dtype=np.float32 if single else np.float64)
            dev = 0
        else:
            dev = 1 if getattr(out, "is_cuda", False) else 0
        nbytes = comps * self.nvox * (4 if single else 8)
        _check(self.lib.rve_get_fields_as(self.h, which, DTYPE_F32 if single else DTYPE_F64, _ptr(out), nbytes, dev),
               self.h)
        return out

    def residuals(self):
        """(e_eq, c_F) arrays of every fixed-point iteration of the latest increment."""
        n = C.c_int(0)
        _check(self.lib.rve_get_residuals(self.h, None, None, 0, C.byref(n)), self.h)
        e = (C.c_double * max(1, n.value))()
        c = (C.c_double * max(1, n.value))()
        _check(self.lib.rve_get_residuals(self.h, e, c, n.value, None), self.h)
        return np.array(e[: n.value]), np.array(c[: n.value])

    def kernel_times(self, reset=False) -> dict:
        """{kernel: (milliseconds, launches)} accumulated with CUDA events (timing=True)."""
        ms = (C.c_double * len(KERNELS))()
        n = (C.c_longlong * len(KERNELS))()
        _check(self.lib.rve_kernel_times(self.h, ms, n, 1 if reset else 0), self.h)
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNELS)}

    def save_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(self.lib.rve_save_state(self.h, None, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(self.lib.rve_save_state(self.h, buf, C.byref(n)), self.h)
        return buf.raw

    def load_state(self, blob: bytes):
        _check(self.lib.rve_load_state(self.h, C.c_char_p(blob), len(blob)), self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.rve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- kernel-level entry points ----------------------------------------------
def step_batch(solvers, n_increments=1) -> int:
    """Advance several RVE solvers by n_increments each, concurrently (rve_step_batch).
    Returns the total fixed-point iterations; raises RVEError naming the first failing
    solver (the others still ran all increments)."""
    solvers = list(solvers)
    if not solvers:
        return 0
    lib = load_library()
    arr = (C.c_void_p * len(solvers))(*[s.h for s in solvers])
    it = C.c_longlong(0)
    failed = C.c_int(-1)
    st = lib.rve_step_batch(arr, len(solvers), int(n_increments), C.byref(it), C.byref(failed))
    if st != 0:
        raise RVEError(st, lib.rve_last_error(None).decode(), index=failed.value)
    return int(it.value)


def batch_grouped(solvers) -> bool:
    """Whether step_batch steps these solvers as one group (one launch per pass over all
    members) rather than on private streams (rve_batch_grouped)."""
    solvers = list(solvers)
    lib = load_library()
    arr = (C.c_void_p * max(1, len(solvers)))(*[s.h for s in solvers])
    out = C.c_int(0)
    st = lib.rve_batch_grouped(arr, len(solvers), C.byref(out))
    if st != 0:
        raise RVEError(st, lib.rve_last_error(None).decode())
    return bool(out.value)


def material_point(R, eps_n, eps, state, dt, n_sub, precision=FP64, **material):
    """One increment of the per-voxel constitutive update on CUDA tensors.

    R (nvox, 9), eps_n/eps (6, nvox), state (34, nvox) updated in place; returns sigma (6, nvox).
    """
    import torch

    lib = load_library()
    m = default_material()
    for k, v in material.items():
        setattr(m, k, float(v))
    sigma = torch.empty_like(eps)
    nvox = eps.shape[1]
    st = lib.rve_material_point(precision, C.byref(m), nvox, _ptr(R), _ptr(eps_n), _ptr(eps), _ptr(state),
                                _ptr(sigma), float(dt), int(n_sub), _torch_stream())
    _check(st, None)
    return sigma


def material_point_vjp(R, eps_n, eps, state, sigma_b, state_b, dt, n_sub, precision=FP64, **material):
    """Reverse pass of `material_point` on CUDA tensors (rve_material_point_vjp).

    state (34, nvox) is the state at t_n (unchanged); state_b (34, nvox) holds the adjoint of
    the state at t_{n+1} and is overwritten with the adjoint of the state at t_n.  Returns
    (eps_b, eps_n_b, R_b (9, nvox), param_b (9, nvox)); param_b rows: r0_ord, r0_sup,
    r0_twin, Q_s, Q_b, b_s, b_b, c, d (per voxel)."""
    import torch

    lib = load_library()
    m = default_material()
    for k, v in material.items():
        setattr(m, k, float(v))
    nvox = eps.shape[1]
    eps_b = torch.empty_like(eps)
    eps_n_b = torch.empty_like(eps)
    R_b = torch.empty((9, nvox), dtype=eps.dtype, device=eps.device)
    param_b = torch.empty((9, nvox), dtype=eps.dtype, device=eps.device)
    st = lib.rve_material_point_vjp(precision, C.byref(m), nvox, _ptr(R), _ptr(eps_n), _ptr(eps), _ptr(state),
                                    _ptr(sigma_b), _ptr(state_b), _ptr(eps_b), _ptr(eps_n_b), _ptr(R_b),
                                    _ptr(param_b), float(dt), int(n_sub), _torch_stream())
    _check(st, None)
    return eps_b, eps_n_b, R_b, param_b


PARAM_NAMES = ["r0_ord", "r0_sup", "r0_twin", "Q_s", "Q_b", "b_s", "b_b", "c", "d"]


def history_storage(n_increments, nvox, checkpoint_every, memory_budget):
    """How history_gradient keeps the history: (store_all, checkpoint_every).

    checkpoint_every = k (an int) is taken as given (checkpoints every k increments).  With
    None, every increment's fields are kept on the device when (n_increments + 1) * 8 *
    (6 + 34) * nvox bytes fit in memory_budget; otherwise checkpoints every
    ceil(sqrt(n_increments)) increments (at least 1)."""
    if checkpoint_every is not None:
        if int(checkpoint_every) < 1:
            raise ValueError("checkpoint_every must be >= 1 or None")
        return False, int(checkpoint_every)
    need = 8 * (6 + 34) * int(nvox) * (int(n_increments) + 1)
    if need <= memory_budget:
        return True, max(1, int(n_increments))
    return False, max(1, math.isqrt(max(int(n_increments) - 1, 0)) + 1)


def history_gradient(grain_id, euler, n_increments, dt, target, weights=None, precision=FP64, material=None,
                     Edot=(0, 0, 1e-3, 0, 0, 0), checkpoint_every=None, memory_budget=None, **options):
    """Misfit J = sum_n w_n (<sigma_zz>_n - target_n)^2 of a load history and its gradient
    with respect to the parameters PARAM_NAMES and every grain's Bunge angles, by the
    adjoint of the history (rve_adjoint_increment).

    The reverse pass needs the strain and state of every increment.  With checkpoint_every
    = None (the default) the forward pass keeps every increment's fields on the device
    (8 (6 + 34) bytes per voxel and increment) when they fit in memory_budget bytes
    (default: half the free device memory), so nothing is replayed; otherwise it
    checkpoints every ceil(sqrt(n_increments)) increments.  With checkpoint_every = k the
    forward pass saves the state every k increments and the reverse pass replays each
    segment from its checkpoint.
    Returns (J, dJ/dparams (9,), dJ/deuler (n_grains, 3), info)."""
    import torch

    lib = load_library()
    material = dict(material or {})
    euler = np.ascontiguousarray(np.asarray(euler, dtype=np.float64))
    target = np.asarray(target, dtype=np.float64)
    w = np.ones(n_increments) if weights is None else np.asarray(weights, dtype=np.float64)

    def make():
        s = RVE(grain_id, euler, precision=precision, **options)
        if material:
            s.set_material(**material)
        s.set_mixed_load(Edot=Edot, dt=dt)
        return s

    dev = torch.device("cuda", options.get("device", 0))
    fwd = make()
    nvox = fwd.nvox

    def fields_of(h):
        eps = h.field(FIELD_STRAIN, out=torch.empty((6,) + h.shape, dtype=torch.float64, device=dev))
        st = torch.cat([h.field(f, out=torch.empty((FIELD_COMPONENTS[f],) + h.shape, dtype=torch.float64,
                                                   device=dev)).reshape(-1, nvox)
                        for f in (FIELD_EPS_P, FIELD_V, FIELD_ALPHA)]).contiguous()
        return eps.reshape(6, nvox).contiguous(), st

    budget = memory_budget
    if checkpoint_every is None and budget is None:
        budget = torch.cuda.mem_get_info(dev)[0] // 2
    store_all, checkpoint_every = history_storage(n_increments, nvox, checkpoint_every, budget)
    ckpt = {0: fwd.save_state()} if not store_all else {}
    stored = [fields_of(fwd)] if store_all else None
    S = []
    for k in range(1, n_increments + 1):
        fwd.step(1)
        S.append(fwd.history()[-1]["S"].copy())
        if store_all:
            stored.append(fields_of(fwd))
        elif k % checkpoint_every == 0 and k < n_increments:
            ckpt[k] = fwd.save_state()
    fwd.close()
    S = np.array(S)
    J = float(np.sum(w * (S[:, 2] - target) ** 2))
    dS = np.zeros((n_increments, 6))
    dS[:, 2] = 2.0 * w * (S[:, 2] - target)
    state_b = torch.zeros((34, nvox), dtype=torch.float64, device=dev)
    eps_b = torch.zeros((6, nvox), dtype=torch.float64, device=dev)
    pgrad = (C.c_double * 9)()
    egrad = (C.c_double * euler.size)()
    adj_iters = C.c_longlong(0)
    adj = make()
    rep = make() if not store_all else None
    starts = [0] if store_all else sorted(ckpt)
    for seg, k0 in reversed(list(enumerate(starts))):
        k1 = starts[seg + 1] if seg + 1 < len(starts) else n_increments
        if store_all:
            fields = stored
        else:
            # replay the segment from its checkpoint, keeping strain and state at k0 .. k1
            rep.load_state(ckpt[k0])
            fields = []
            for k in range(k0, k1 + 1):
                if k > k0:
                    rep.step(1)
                fields.append(fields_of(rep))
        for k in range(k1, k0, -1):
            e_prev, s_prev = fields[k - 1 - k0]
            e_cur, _ = fields[k - k0]
            d6 = (C.c_double * 6)(*dS[k - 1])
            _check(lib.rve_adjoint_increment(adj.h, _ptr(e_prev), _ptr(e_cur), _ptr(s_prev), d6, float(dt),
                                             _ptr(state_b), _ptr(eps_b), pgrad, egrad, C.byref(adj_iters)), adj.h)
    adj.close()
    if rep is not None:
        rep.close()
    info = {"S": S, "adjoint_iterations": int(adj_iters.value), "checkpoints": [] if store_all else starts,
            "stored_fields": store_all}
    return J, np.array(pgrad[:]), np.array(egrad[:]).reshape(euler.shape), info


class HistoryMisfit:
    """torch.autograd.Function for the load-history misfit: apply(params (9,), euler
    (n_grains, 3), config dict) -> J, with the adjoint gradient in backward.  `config`
    holds grain_id, n_increments, dt, target and optional weights, precision, material,
    Edot, checkpoint_every and solver options."""

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, params, euler, config):
                mat = dict(config.get("material", {}))
                mat.update({k: float(v) for k, v in zip(PARAM_NAMES, params.detach().cpu().tolist())})
                cfg = {k: v for k, v in config.items() if k not in ("grain_id", "n_increments", "dt", "target",
                                                                   "material")}
                J, gp, ge, _ = history_gradient(config["grain_id"], euler.detach().cpu().numpy(),
                                                config["n_increments"], config["dt"], config["target"],
                                                material=mat, **cfg)
                ctx.save_for_backward(torch.as_tensor(gp, dtype=params.dtype),
                                      torch.as_tensor(ge, dtype=euler.dtype))
                return torch.tensor(J, dtype=params.dtype)

            @staticmethod
            def backward(ctx, g):
                gp, ge = ctx.saved_tensors
                return g * gp, g * ge, None

        return _F

    @classmethod
    def apply(cls, params, euler, config):
        return cls._fn().apply(params, euler, config)


def alu_probe(kind, blocks, iters, sink):
    """Enqueue one ALU throughput probe (rve_alu_probe) on torch's current stream; `sink`
    is a CUDA tensor of at least 8 bytes.  Returns the operations of the launch."""
    lib = load_library()
    ops = C.c_double(0.0)
    _check(lib.rve_alu_probe(int(kind), int(blocks), int(iters), _ptr(sink), _torch_stream(), C.byref(ops)))
    return ops.value


def fft_r2c(real, precision=FP64):
    """Forward 3-D R2C transform of (ncomp, nz, ny, nx) CUDA tensor -> (ncomp, nz, ny, nx//2+1) complex."""
    import torch

    lib = load_library()
    ncomp, nz, ny, nx = real.shape
    cdt = torch.complex128 if precision == FP64 else torch.complex64
    out = torch.empty((ncomp, nz, ny, nx // 2 + 1), dtype=cdt, device=real.device)
    _check(lib.rve_fft_r2c(precision, nx, ny, nz, ncomp, _ptr(real.contiguous()), _ptr(out), _torch_stream()))
    return out


def fft_c2r(spec, nx, precision=FP64):
    """Unnormalised inverse of fft_r2c; `spec` is consumed (overwritten)."""
    import torch

    lib = load_library()
    ncomp, nz, ny, _ = spec.shape
    rdt = torch.float64 if precision == FP64 else torch.float32
    out = torch.empty((ncomp, nz, ny, nx), dtype=rdt, device=spec.device)
    _check(lib.rve_fft_c2r(precision, nx, ny, nz, ncomp, _ptr(spec), _ptr(out), _torch_stream()))
    return out


def label_voronoi(inputs, out=None):
    """Grain-ID map of an inputs.RVEInputs, computed on the GPU; numpy (nz, ny, nx) uint32
    unless `out` (a CUDA int32 tensor) is given."""
    lib = load_library()
    nz, ny, nx = inputs.shape
    seeds = np.ascontiguousarray(inputs.seeds, dtype=np.float64)
    tw = np.ascontiguousarray(inputs.twinned, dtype=np.uint8)
    nrm = np.ascontiguousarray(inputs.twin_normal, dtype=np.float64)
    if out is None:
        res = np.empty((nz, ny, nx), dtype=np.uint32)
        st = lib.rve_label_voronoi(nx, ny, nz, seeds.shape[0], _ptr(seeds), _ptr(tw), _ptr(nrm), _ptr(res), 0, None)
    else:
        res = out
        st = lib.rve_label_voronoi(nx, ny, nz, seeds.shape[0], _ptr(seeds), _ptr(tw), _ptr(nrm), _ptr(res), 1,
                                   _torch_stream())
    _check(st, None)
    return res


def label_voronoi_noalloc(inputs, out):
    """Grain-ID map of an inputs.RVEInputs written into `out`, a CUDA int32 tensor
    (nz, ny, nx), by the entry point that allocates no device memory (its scratch is a
    fixed static array: at most NOALLOC_MAX_PARENTS parents)."""
    import torch

    lib = load_library()
    nz, ny, nx = inputs.shape
    seeds = np.ascontiguousarray(inputs.seeds, dtype=np.float64)
    tw = np.ascontiguousarray(inputs.twinned, dtype=np.uint8)
    nrm = np.ascontiguousarray(inputs.twin_normal, dtype=np.float64)
    if not getattr(out, "is_cuda", False) or tuple(out.shape) != (nz, ny, nx):
        raise ValueError("out must be a CUDA tensor of shape (nz, ny, nx)")
    if out.dtype != torch.int32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous torch.int32 tensor")
    # the library looks up its scratch and takes the stream on the current device: make
    # it the output's device
    with torch.cuda.device(out.device):
        st = lib.rve_label_voronoi_noalloc(nx, ny, nz, seeds.shape[0], _ptr(seeds), _ptr(tw), _ptr(nrm), _ptr(out),
                                           C.c_void_p(torch.cuda.current_stream(out.device).cuda_stream))
    _check(st, None)
    return out
