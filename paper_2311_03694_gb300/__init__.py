"""Python binding of libgrom.so, the GB300 Galerkin ROM engine (include/grom.h).

Argument marshalling only: every step of the contraction and of the reduced
time-stepper runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams; numpy arrays are accepted where the ABI takes host or
device pointers.  There is no CPU fallback: without the built library every
call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build_mod

GROM_OK = 0
GROM_ERR_INVALID_ARG = 1
ERRORS = {
    1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NONFINITE", 5: "TIMEOUT", 6: "BUDGET", 7: "UNSUPPORTED",
}
FORMS = {"full": 0, "cp": 1, "cp_skew": 2, "svd": 3}
STORAGE = {"f64": 0, "f32x2": 1, "f32": 2, "bf16": 3}
STORAGE_BYTES = {"f64": 8, "f32x2": 8, "f32": 4, "bf16": 2}
LAYOUTS = {"dense": 0, "skew_packed": 1}


class _Request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("horizon", ctypes.c_int32), ("arrival", ctypes.c_double),
                ("u0", ctypes.c_void_p), ("u_final", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("trajectory_steps", ctypes.c_int64), ("quanta", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("peak_bytes", ctypes.c_int64), ("peak_active", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("kernel", ctypes.c_int32), ("tile_m", ctypes.c_int32),
                ("split_a", ctypes.c_int32), ("split_b", ctypes.c_int32), ("timed", ctypes.c_int32),
                ("ms", ctypes.c_float), ("ms_rule", ctypes.c_float)]


KERNELS = {"auto": 0, "stream": 1, "tensor": 2}
_KERNEL_NAMES = {v: k for k, v in KERNELS.items()}


def _tuning_dict(t):
    return {"batch": t.batch, "kernel": _KERNEL_NAMES.get(t.kernel, t.kernel), "tile_m": t.tile_m,
            "split_a": t.split_a, "split_b": t.split_b, "timed": t.timed, "ms": t.ms, "ms_rule": t.ms_rule}


def _tuning_struct(d):
    t = _Tuning()
    t.batch, t.kernel = int(d["batch"]), KERNELS[d["kernel"]]
    t.tile_m, t.split_a, t.split_b = int(d.get("tile_m", 0)), int(d.get("split_a", 0)), int(d.get("split_b", 0))
    return t


class GromError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code
        self.name = ERRORS.get(code, str(code))


class _Desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("form", ctypes.c_int32), ("rank", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("tensor", ctypes.c_void_p), ("fa", ctypes.c_void_p), ("fb", ctypes.c_void_p), ("fc", ctypes.c_void_p),
        ("stiffness", ctypes.c_void_p), ("stiffness_diag", ctypes.c_void_p),
        ("mass", ctypes.c_void_p), ("mass_diag", ctypes.c_void_p),
        ("linear", ctypes.c_void_p), ("linear_diag", ctypes.c_void_p), ("forcing", ctypes.c_void_p),
        ("nu", ctypes.c_double), ("dt", ctypes.c_double), ("order", ctypes.c_int32),
        ("defer_tensor", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("layout", ctypes.c_int32),
        ("augmented", ctypes.c_int32), ("no_tile_copy", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


_lib = None

EXPORTS = {
    "grom_create": ([ctypes.POINTER(_Desc), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "grom_upload_tensor_slab": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int32),
    "grom_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "grom_max_n": ([ctypes.c_int32, ctypes.c_int32], ctypes.c_int32),
    "grom_nonlinear": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "grom_traj_create": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
                         ctypes.c_int32),
    "grom_traj_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "grom_step": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "grom_traj_status": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int32),
    "grom_get_state": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "grom_set_state": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "grom_sync": ([ctypes.c_void_p], ctypes.c_int32),
    "grom_rom_bytes": ([ctypes.c_void_p], ctypes.c_int64),
    "grom_step_host": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "grom_set_kernel": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int32),
    "grom_tune_space": ([ctypes.c_int32] * 8 + [ctypes.POINTER(_Tuning), ctypes.c_int32], ctypes.c_int32),
    "grom_autotune": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_Tuning)], ctypes.c_int32),
    "grom_set_tuning": ([ctypes.c_void_p, ctypes.POINTER(_Tuning)], ctypes.c_int32),
    "grom_get_tuning": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_Tuning)], ctypes.c_int32),
    "grom_profile_enable": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int32),
    "grom_profile_read": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
                          ctypes.c_int32),
    "grom_nonlinear_full_noalloc": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "grom_nonlinear_full_noalloc_status": ([ctypes.c_void_p], ctypes.c_int32),
    "grom_server_create": ([ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
                           ctypes.c_int32),
    "grom_server_add_rom": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
                            ctypes.c_int32),
    "grom_server_add_simulated": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_int32)], ctypes.c_int32),
    "grom_serve": ([ctypes.c_void_p, ctypes.POINTER(_Request), ctypes.c_int32, ctypes.POINTER(_Result),
                    ctypes.POINTER(_Stats)], ctypes.c_int32),
    "grom_server_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "grom_selftest_timeout": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int32),
    "grom_last_error": ([], ctypes.c_char_p),
    "grom_als_create": ([ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
                        ctypes.c_int32),
    "grom_als_fit": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                      ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p], ctypes.c_int32),
    "grom_als_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "grom_als_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int32),
}


def lib_path():
    return _build_mod.LIB


def build(force=False, verbose=False):
    """Compile the CUDA library for sm_103a (see build.py)."""
    return _build_mod.build(force=force, verbose=verbose)


def load(path=None):
    """Load libgrom.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = path or lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libgrom.so is not built (call paper_2311_03694_gb300.build())")
        lib = ctypes.CDLL(path)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(code):
    if code != GROM_OK:
        raise GromError(code, load().grom_last_error().decode())


def _ptr(x):
    """Pointer of a numpy array (host) or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags.c_contiguous, "need a contiguous float64 array"
        return x.ctypes.data
    assert str(x.dtype) == "torch.float64" and x.is_contiguous(), "need a contiguous float64 tensor"
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def max_n(form, storage):
    return load().grom_max_n(FORMS[form], STORAGE[storage])


def tune_space(form, storage, n, batch, max_batch=None, rank=0, layout="dense", sm_count=152):
    """The configurations the autotuner times for `batch` trajectories of such a
    ROM (grom_tune_space; host arithmetic only): the rules' first."""
    lib = load()
    args = (FORMS[form], STORAGE[storage], LAYOUTS[layout], int(n), int(rank),
            int(max_batch if max_batch is not None else batch), int(batch), int(sm_count))
    count = lib.grom_tune_space(*args, None, 0)
    if count < 0:
        raise GromError(1, "grom_tune_space: invalid arguments")
    buf = (_Tuning * max(count, 1))()
    lib.grom_tune_space(*args, buf, count)
    return [_tuning_dict(buf[i]) for i in range(count)]


def stored_row_bytes(n, storage):
    """Bytes of one stored row (i, j) of the dense layout: round_up(n, 64)
    elements of the storage type (F32X2: a hi and a lo plane of floats)."""
    return (int(n) + 63) // 64 * 64 * STORAGE_BYTES[storage]


def nonlinear_full_noalloc(n, storage, tensor, u, c, stream=None):
    """grom_nonlinear_full_noalloc: c = C(u)u for one trajectory without any
    library allocation.  tensor is a device tensor already in the stored
    layout (see include/grom.h and stored_layout()); u, c are float64 device
    tensors of n entries.  The C entry point cannot see the extent of the
    caller's buffers, so they are checked here: every operand on the current
    device, tensor holding n*n stored rows, u and c n entries each."""
    import torch

    n = int(n)
    if storage not in STORAGE:
        raise GromError(GROM_ERR_INVALID_ARG, "unknown storage %r" % (storage,))
    dev = torch.cuda.current_device()
    for name, x in (("tensor", tensor), ("u", u), ("c", c)):
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.device.index != dev:
            raise GromError(GROM_ERR_INVALID_ARG, "%s must be a tensor on cuda:%d" % (name, dev))
    if not tensor.is_contiguous():
        raise GromError(GROM_ERR_INVALID_ARG, "tensor must be contiguous")
    need = n * n * stored_row_bytes(max(n, 1), storage)
    if tensor.numel() * tensor.element_size() < need:
        raise GromError(GROM_ERR_INVALID_ARG, "tensor holds %d bytes, the stored layout of n=%d %s needs %d"
                        % (tensor.numel() * tensor.element_size(), n, storage, need))
    for name, x in (("u", u), ("c", c)):
        if x.numel() != n:
            raise GromError(GROM_ERR_INVALID_ARG, "%s has %d entries, n = %d" % (name, x.numel(), n))
    _check(load().grom_nonlinear_full_noalloc(n, STORAGE[storage], tensor.data_ptr(), _ptr(u), _ptr(c),
                                              ctypes.c_void_p(_stream_handle(stream))))
    return c


def nonlinear_full_noalloc_status(stream=None):
    """grom_nonlinear_full_noalloc_status: raises GromError (GROM_ERR_TIMEOUT)
    when a device wait of the last allocation-free call on this device gave
    up; synchronises the stream."""
    _check(load().grom_nonlinear_full_noalloc_status(ctypes.c_void_p(_stream_handle(stream))))


def stored_layout(C, storage):
    """The stored device layout of a dense FP64 torch tensor C (n, n, n):
    k padded with zeros to a multiple of 64, converted to the storage type
    (F32X2 rows are [hi | lo]).  Returns a flat uint8 view of the bytes."""
    import torch

    n = C.shape[0]
    np_ = (n + 63) // 64 * 64
    P = torch.zeros((n, n, np_), dtype=torch.float64, device=C.device)
    P[:, :, :n] = C
    if storage == "f64":
        out = P
    elif storage == "f32":
        out = P.to(torch.float32)
    elif storage == "bf16":
        # one round-to-nearest-even from FP64 to the 8-bit significand (the
        # library's rounding; a cast through FP32 would round twice): round
        # the FP64 bit pattern at bit 45, after which the FP32 and BF16
        # conversions are exact
        bits = P.view(torch.int64)
        bits = (bits + ((1 << 44) - 1) + ((bits >> 45) & 1)) & ~((1 << 45) - 1)
        out = bits.view(torch.float64).to(torch.float32).to(torch.bfloat16)
    elif storage == "f32x2":
        hi = P.to(torch.float32)
        lo = (P - hi.to(torch.float64)).to(torch.float32)
        out = torch.cat([hi, lo], dim=2)
    else:
        raise ValueError(storage)
    return out.contiguous().view(torch.uint8).reshape(-1)


class Rom:
    """A reduced-order model on the GPU (wraps grom_create / grom_destroy).

    form: "full" (tensor n^3), "cp" (factors A, B, C), "cp_skew" (U, V, W) or
    "svd" (factors (U, sigma, V): U n x rank, sigma rank, V n x rank x n).
    storage: "f64", "f32x2", "f32" or "bf16".  stiffness may be a length-n
    diagonal or an n x n matrix; mass None means identity.
    layout (full and svd forms): "dense" or "skew_packed" (one entry of each
    pair C_ijk = -C_kji stored; the tensor, or each V slice, must be skew).
    augmented: the operator includes the zeroth mode (full: tensor n x (n+1)
    x (n+1); cp: fb and fc with n+1 rows); see grom_desc.augmented.
    tile_copy: dense BF16 full form with max_batch > 8 keeps a tile-major copy
    of the tensor for the tensor-core kernel (False: row layout only, less
    memory); see grom_desc.no_tile_copy.
    """

    def __init__(self, n, form="full", storage="f64", tensor=None, factors=None, stiffness=None, mass=None,
                 linear=None, forcing=None, nu=1e-2, dt=1e-3, order=3, max_batch=1, defer_tensor=False,
                 stream=None, layout="dense", augmented=False, tile_copy=True):
        lib = load()
        keep = []

        def arr(x):
            if x is None:
                return None
            if isinstance(x, np.ndarray):
                x = np.ascontiguousarray(x, dtype=np.float64)
            keep.append(x)
            return _ptr(x)

        d = _Desc()
        d.n, d.form, d.storage = int(n), FORMS[form], STORAGE[storage]
        d.nu, d.dt, d.order, d.max_batch = float(nu), float(dt), int(order), int(max_batch)
        d.defer_tensor = 1 if defer_tensor else 0
        d.layout = LAYOUTS[layout]
        d.augmented = 1 if augmented else 0
        d.no_tile_copy = 0 if tile_copy else 1
        if form == "full":
            d.tensor = arr(tensor)
        else:
            fa, fb, fc = factors
            d.rank = int(fa.shape[1])
            d.fa, d.fb, d.fc = arr(fa), arr(fb), arr(fc)
        if stiffness is None:
            raise ValueError("stiffness is required")
        if np.ndim(stiffness) == 1:
            d.stiffness_diag = arr(stiffness)
        else:
            d.stiffness = arr(stiffness)
        if mass is not None:
            if np.ndim(mass) == 1:
                d.mass_diag = arr(mass)
            else:
                d.mass = arr(mass)
        if linear is not None:
            if np.ndim(linear) == 1:
                d.linear_diag = arr(linear)
            else:
                d.linear = arr(linear)
        d.forcing = arr(forcing)
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(lib.grom_create(ctypes.byref(d), ctypes.c_void_p(self._stream), ctypes.byref(h)))
        self._h = h
        self.n, self.form, self.storage, self.max_batch = int(n), form, storage, int(max_batch)
        self.layout = layout
        self.rank = int(d.rank)
        self.order = int(order)

    @property
    def handle(self):
        return self._h

    def upload_slab(self, i0, rows):
        _check(load().grom_upload_tensor_slab(self._h, int(i0), int(i0) + rows.shape[0], _ptr(rows)))

    def nonlinear(self, u, c):
        """c = C(u)u for device tensors u, c of shape (batch, n), float64."""
        batch = 1 if u.dim() == 1 else u.shape[0]
        _check(load().grom_nonlinear(self._h, batch, _ptr(u), _ptr(c)))
        return c

    def sync(self):
        _check(load().grom_sync(self._h))

    def selftest_timeout(self, limit_ns):
        """Run a bounded device wait that nothing signals (see grom_selftest_timeout)."""
        _check(load().grom_selftest_timeout(self._h, int(limit_ns)))

    def set_kernel(self, kernel):
        """Override the contraction kernel: "auto", "stream" (the SIMT streaming or CP
        kernels, one launch per step) or "tensor" (the tcgen05 kernels: K2, K2P, K3T)."""
        _check(load().grom_set_kernel(self._h, KERNELS[kernel]))

    def autotune(self, batch, reps=0):
        """Time the kernel choices and tile shapes for `batch` trajectories and
        keep the fastest for its batch bucket (grom_autotune); returns the entry
        installed, a dict that set_tuning accepts in a later run."""
        t = _Tuning()
        _check(load().grom_autotune(self._h, int(batch), int(reps), ctypes.byref(t)))
        return _tuning_dict(t)

    def set_tuning(self, entry):
        """Install an entry (a dict from autotune or tune_space); kernel "auto" removes it."""
        _check(load().grom_set_tuning(self._h, ctypes.byref(_tuning_struct(entry))))

    def get_tuning(self, batch):
        t = _Tuning()
        _check(load().grom_get_tuning(self._h, int(batch), ctypes.byref(t)))
        return _tuning_dict(t)

    def profile(self, enable=True):
        _check(load().grom_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """(summed device ms, launches) of the main contraction kernel since enable."""
        ms, cnt = ctypes.c_double(), ctypes.c_int64()
        _check(load().grom_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    @property
    def nbytes(self):
        return load().grom_rom_bytes(self._h)

    def close(self):
        if getattr(self, "_h", None):
            _check(load().grom_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Trajectories:
    """A batch of trajectories of one Rom (grom_traj_*)."""

    def __init__(self, rom, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64) if isinstance(u0, np.ndarray) else u0
        self.batch = 1 if u0.ndim == 1 else u0.shape[0]
        self.rom = rom
        h = ctypes.c_void_p()
        _check(load().grom_traj_create(rom.handle, self.batch, _ptr(u0), ctypes.byref(h)))
        self._h = h

    def step(self, nsteps, energy=None, invariant=None):
        _check(load().grom_step(self._h, int(nsteps), _ptr(energy), _ptr(invariant)))

    def step_host(self, nsteps, u_in=None, u_out=None):
        """grom_step_host: feed u_in (optional), step, copy the new state to u_out."""
        _check(load().grom_step_host(self._h, int(nsteps), _ptr(u_in), _ptr(u_out)))

    def status(self):
        bad = ctypes.c_int32(-1)
        code = load().grom_traj_status(self._h, ctypes.byref(bad))
        if code not in (GROM_OK, 4):
            _check(code)
        return code, bad.value

    def get_state(self):
        out = np.empty((self.batch, 6 * self.rom.n + 1))
        _check(load().grom_get_state(self._h, out.ctypes.data))
        return out

    def set_state(self, hist):
        hist = np.ascontiguousarray(hist, dtype=np.float64).reshape(self.batch, 6 * self.rom.n + 1)
        _check(load().grom_set_state(self._h, hist.ctypes.data))

    def close(self):
        if getattr(self, "_h", None):
            _check(load().grom_traj_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Als:
    """CP fitting context (grom_als_create / grom_als_fit / grom_als_destroy)."""

    METHODS = {"plain": 0, "skew": 1}

    def __init__(self, tensor, stream=None):
        n = int(tensor.shape[0])
        if isinstance(tensor, np.ndarray):
            tensor = np.ascontiguousarray(tensor, dtype=np.float64)
        self._keep = tensor
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(load().grom_als_create(n, _ptr(tensor), ctypes.c_void_p(self._stream), ctypes.byref(h)))
        self._h = h
        self.n = n

    def fit(self, factors, iters, method="plain", lam=0.5, subiters=1, ridge=0.0):
        """Runs `iters` iterations from `factors` ((A1, A2, A3) for "plain",
        (A1, B1) for "skew"); returns the new factors and the residuals."""
        fs = [np.array(f, dtype=np.float64, order="C") for f in factors]
        rank = fs[0].shape[1]
        res = np.empty(iters)
        fc = _ptr(fs[2]) if len(fs) > 2 else None
        _check(load().grom_als_fit(self._h, int(rank), self.METHODS[method], int(iters), float(lam), int(subiters),
                                   float(ridge), _ptr(fs[0]), _ptr(fs[1]), fc, _ptr(res)))
        return fs, res

    def stats(self):
        """(MTTKRP device ms, MTTKRP launches, SPD solve ms) since the last call."""
        ms, calls, solve = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(load().grom_als_stats(self._h, ctypes.byref(ms), ctypes.byref(calls), ctypes.byref(solve)))
        return ms.value, calls.value, solve.value

    def close(self):
        if getattr(self, "_h", None):
            load().grom_als_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over resident ROMs (grom_server_*, grom_serve).

    simulate=True runs the scheduler without a GPU (models added with
    add_simulated cost step_seconds of virtual time per batched step).
    """

    def __init__(self, budget_bytes, quantum=16, simulate=False):
        h = ctypes.c_void_p()
        _check(load().grom_server_create(int(budget_bytes), int(quantum), 1 if simulate else 0, ctypes.byref(h)))
        self._h = h
        self._roms = []
        self.n = []

    def add_rom(self, rom, max_slots):
        mid = ctypes.c_int32()
        _check(load().grom_server_add_rom(self._h, rom.handle, int(max_slots), ctypes.byref(mid)))
        self._roms.append(rom)
        self.n.append(rom.n)
        return mid.value

    def add_simulated(self, n, rom_bytes, max_slots, step_seconds):
        mid = ctypes.c_int32()
        _check(load().grom_server_add_simulated(self._h, int(n), int(rom_bytes), int(max_slots), float(step_seconds),
                                                ctypes.byref(mid)))
        self.n.append(int(n))
        return mid.value

    def serve(self, models, horizons, arrivals, u0s, want_final=False):
        """Run requests (model id, horizon, arrival time, initial state) to completion.

        Returns a dict of numpy arrays (status, steps, t_admit, t_done), the
        final states when want_final, and the run statistics."""
        count = len(models)
        reqs = (_Request * max(count, 1))()
        finals = []
        keep = []
        for q in range(count):
            u0 = np.ascontiguousarray(u0s[q], dtype=np.float64)
            keep.append(u0)
            reqs[q].model, reqs[q].horizon, reqs[q].arrival = int(models[q]), int(horizons[q]), float(arrivals[q])
            reqs[q].u0 = u0.ctypes.data
            if want_final:
                f = np.empty(self.n[int(models[q])])
                finals.append(f)
                reqs[q].u_final = f.ctypes.data
        res = (_Result * max(count, 1))()
        st = _Stats()
        _check(load().grom_serve(self._h, reqs, count, res, ctypes.byref(st)))
        out = {k: np.array([getattr(res[q], k) for q in range(count)]) for k in ("status", "steps", "t_admit", "t_done")}
        out["final"] = finals
        out["stats"] = {k: getattr(st, k) for k in ("trajectory_steps", "quanta", "seconds", "peak_bytes",
                                                    "peak_active")}
        return out

    def close(self):
        if getattr(self, "_h", None):
            _check(load().grom_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
