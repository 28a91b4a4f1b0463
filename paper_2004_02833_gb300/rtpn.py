"""Thin ctypes binding of librtpn.so (include/rtpn.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts numpy arrays (host)
and torch tensors (host or device) into pointers, dtypes and memory kinds, and raises on a
non-zero status.  There is no fallback: if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "librtpn.so")

OK, EINVAL, ECFL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
BC = {"periodic": 0, "vacuum": 1}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
DTYPE_F64, DTYPE_F32 = 0, 1
HOST, DEVICE = 0, 1
KERNEL = {"auto": 0, "generic": 1, "window": 2, "stage": 3, "fused": 4}


class RtpnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rtpn error {code}: {msg}")
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n_c", ctypes.c_int), ("n_even", ctypes.c_int),
                ("n_odd", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("bc", ctypes.c_int), ("precision", ctypes.c_int),
                ("kernel", ctypes.c_int), ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("state_bytes", ctypes.c_size_t), ("factor_bytes", ctypes.c_size_t),
                ("steps_done", ctypes.c_longlong), ("tile", ctypes.c_int * 3), ("depth", ctypes.c_int),
                ("hy", ctypes.c_double), ("hz", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); every name here is declared in include/rtpn.h
SIGNATURES = {
    "rtpn_version": (_I, []),
    "rtpn_strerror": (ctypes.c_char_p, [_I]),
    "rtpn_component_info": (_I, [_I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rtpn_coupling_dense": (_I, [_I, _I, _P]),
    "rtpn_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _D, _I, _I, _D]),
    "rtpn_destroy": (_I, [_P]),
    "rtpn_set_stream": (_I, [_P, _P]),
    "rtpn_set_spacing": (_I, [_P, _D, _D, _D]),
    "rtpn_set_scattering": (_I, [_P, _P, _I]),
    "rtpn_set_kernel": (_I, [_P, _I, _I, _I, _I]),
    "rtpn_set_kernel_ex": (_I, [_P, _I, _I, _I, _I, _I]),
    "rtpn_set_media": (_I, [_P, _P, _P, _P, _I, _I]),
    "rtpn_set_moments": (_I, [_P, _P, _I, _I]),
    "rtpn_get_moments": (_I, [_P, _P, _I, _I]),
    "rtpn_set_component": (_I, [_P, _I, _P, _I, _I]),
    "rtpn_get_component": (_I, [_P, _I, _P, _I, _I]),
    "rtpn_zero_moments": (_I, [_P]),
    "rtpn_step": (_I, [_P, _I]),
    "rtpn_substep": (_I, [_P, _I, _I]),
    "rtpn_copy_planes": (_I, [_P, _I, _P, _I, _I, _I]),
    "rtpn_sum_u0": (_I, [_P, ctypes.POINTER(_D)]),
    "rtpn_count_nonfinite": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "rtpn_sum_static": (_I, [_P, _I, ctypes.c_longlong, _P, _P]),
    "rtpn_synchronize": (_I, [_P]),
    "rtpn_test_wait_timeout": (_I, [_P, _I, ctypes.c_longlong]),
    "rtpn_adjoint": (_I, [_P, _P, _I, _I, _I, _I, _P, _P, _P, _I, ctypes.POINTER(_D)]),
    "rtpn_adjoint_release": (_I, [_P]),
    "rtpn_detector": (_I, [_P, _P, _I, _I, _P, _I]),
    "rtpn_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P, _P, _P, _I]),
    "rtpn_batch_destroy": (_I, [_P]),
    "rtpn_batch_count": (_I, [_P]),
    "rtpn_batch_instance": (_P, [_P, _I]),
    "rtpn_batch_set_stream": (_I, [_P, _P]),
    "rtpn_batch_set_tile": (_I, [_P, _I, _I, _I]),
    "rtpn_batch_get_tile": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rtpn_batch_step": (_I, [_P, _I]),
    "rtpn_batch_step_looped": (_I, [_P, _I]),
    "rtpn_batch_synchronize": (_I, [_P]),
    "rtpn_batch_last_error": (ctypes.c_char_p, [_P]),
    "rtpn_autotune": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "rtpn_batch_autotune": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "rtpn_get_info": (_I, [_P, ctypes.POINTER(Info)]),
    "rtpn_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load librtpn.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2004_02833_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != OK:
        msg = lib().rtpn_last_error(ctx).decode() if ctx is not None else ""
        raise RtpnError(rc, msg or lib().rtpn_strerror(rc).decode())


def _buf(x, want_dtype=None):
    """(pointer, dtype code, where, keepalive) for a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype not in (np.float64, np.float32):
            x = x.astype(np.float64)
        x = np.ascontiguousarray(x)
        code = DTYPE_F64 if x.dtype == np.float64 else DTYPE_F32
        return x.ctypes.data, code, HOST, x
    import torch  # only for tensors the caller already holds

    if not isinstance(x, torch.Tensor):
        return _buf(np.asarray(x, dtype=np.float64))
    if x.dtype not in (torch.float64, torch.float32):
        raise TypeError("tensors must be float64 or float32")
    if not x.is_contiguous():
        raise ValueError("tensors must be contiguous")
    code = DTYPE_F64 if x.dtype == torch.float64 else DTYPE_F32
    return x.data_ptr(), code, (DEVICE if x.is_cuda else HOST), x


def component_info(N: int, c: int):
    """(l, m, (gx, gy, gz), class) of interface component c."""
    l, m, cls = _I(), _I(), _I()
    slots = (_I * 3)()
    _check(lib().rtpn_component_info(N, c, ctypes.byref(l), ctypes.byref(m), slots,
                                     ctypes.byref(cls)))
    return l.value, m.value, tuple(slots), cls.value


def coupling_dense(N: int, axis: int) -> np.ndarray:
    n = (N + 1) ** 2
    out = np.zeros((n, n), dtype=np.float64)
    _check(lib().rtpn_coupling_dense(N, axis, out.ctypes.data))
    return out


def sum_static(x, out, stream=None):
    """FP64 sum of the device tensor x (float32/float64) into the one-element device float64 tensor
    out, without any allocation by the library (see rtpn_sum_static in include/rtpn.h)."""
    import torch

    # checked before anything reaches the library: the kernel reads x.numel() values of 4 or 8 bytes
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError(f"sum_static sums float32 or float64 tensors, not {x.dtype}")
    if out.dtype != torch.float64 or out.numel() < 1:
        raise ValueError("out must hold at least one float64 value")
    if not (x.is_cuda and out.is_cuda and x.is_contiguous()):
        raise ValueError("x must be a contiguous CUDA tensor and out a CUDA tensor")
    code = DTYPE_F64 if x.dtype == torch.float64 else DTYPE_F32
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    rc = lib().rtpn_sum_static(_P(x.data_ptr()), code, x.numel(), _P(out.data_ptr()), _P(handle or 0))
    if rc != OK:
        raise RtpnError(rc, lib().rtpn_last_error(None).decode() or lib().rtpn_strerror(rc).decode())
    return out


class Context:
    """One P_N problem on the current CUDA device (owns its device memory)."""

    def __init__(self, N: int, shape, h: float, bc: str = "periodic", precision: str = "fp32",
                 dt: float | None = None):
        nz, ny, nx = shape
        p = _P()
        rc = lib().rtpn_create(ctypes.byref(p), N, nx, ny, nz, float(h), BC[bc],
                               PRECISION[precision], float(dt or 0.0))
        if rc != OK:
            raise RtpnError(rc, lib().rtpn_last_error(None).decode())
        self._p = p
        self.N, self.shape, self.h, self.bc, self.precision = N, tuple(shape), h, bc, precision
        self.n_c = (N + 1) ** 2

    # -- life cycle
    def close(self):
        if getattr(self, "_p", None):
            lib().rtpn_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, rc):
        _check(rc, self._p)

    # -- configuration
    def set_scattering(self, f=None):
        """Anisotropic scattering moments f_l = Sigma_sl / sigma_s, l = 0..N (f_0 = 1); None restores
        isotropic scattering.  Runs on the generic kernel, and on the window kernel up to N = 15."""
        if f is None:
            self._chk(lib().rtpn_set_scattering(self._p, None, 0))
            return
        arr = np.ascontiguousarray(f, dtype=np.float64)
        self._chk(lib().rtpn_set_scattering(self._p, arr.ctypes.data_as(_P), int(arr.size)))

    def set_spacing(self, hx: float, hy: float, hz: float):
        """Cell sizes along x, y and z (non-cubic cells run on the staged and generic kernels)."""
        self._chk(lib().rtpn_set_spacing(self._p, float(hx), float(hy), float(hz)))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (the context's own stream)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._chk(lib().rtpn_set_stream(self._p, _P(handle or 0)))

    def set_kernel(self, kernel: str = "auto", tile=(0, 0, 0), depth: int = 0):
        self._chk(lib().rtpn_set_kernel_ex(self._p, KERNEL[kernel], *tile, int(depth)))

    def autotune(self, reps: int = 2):
        """Time candidate window-kernel tiles on this context's data, apply the best; (tile, ms)."""
        tile = (_I * 3)()
        ms = _D()
        self._chk(lib().rtpn_autotune(self._p, int(reps), tile, ctypes.byref(ms)))
        return tuple(tile), ms.value

    def info(self) -> Info:
        out = Info()
        self._chk(lib().rtpn_get_info(self._p, ctypes.byref(out)))
        return out

    # -- data
    def set_media(self, sigma_a, sigma_s, q):
        bufs = [_buf(a) for a in (sigma_a, sigma_s, q)]
        codes = {b[1] for b in bufs}
        wheres = {b[2] for b in bufs}
        if len(codes) != 1 or len(wheres) != 1:
            raise ValueError("media arrays must share dtype and memory kind")
        self._chk(lib().rtpn_set_media(self._p, bufs[0][0], bufs[1][0], bufs[2][0],
                                       codes.pop(), wheres.pop()))

    def set_moments(self, u):
        ptr, code, where, keep = _buf(u)
        self._chk(lib().rtpn_set_moments(self._p, ptr, code, where))

    def get_moments(self, out=None):
        """Full state [c, z, y, x] in interface order; into `out` (array/tensor) or a new FP64 array."""
        if out is None:
            out = np.empty((self.n_c,) + self.shape, dtype=np.float64)
        ptr, code, where, keep = _buf(out)
        self._chk(lib().rtpn_get_moments(self._p, ptr, code, where))
        return out

    def set_component(self, c: int, field):
        ptr, code, where, keep = _buf(field)
        self._chk(lib().rtpn_set_component(self._p, c, ptr, code, where))

    def get_component(self, c: int, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, code, where, keep = _buf(out)
        self._chk(lib().rtpn_get_component(self._p, c, ptr, code, where))
        return out

    def zero_moments(self):
        self._chk(lib().rtpn_zero_moments(self._p))

    # -- compute
    def step(self, k: int = 1):
        self._chk(lib().rtpn_step(self._p, int(k)))

    def substep(self, cls: int, half: bool = False):
        """One pass S^cls_tau (tau = dt, or dt/2 with half=True; odd class only)."""
        self._chk(lib().rtpn_substep(self._p, int(cls), int(bool(half))))

    _pass = substep

    def adjoint(self, w, k: int, ckpt_every: int = 20, out=None):
        """J = sum w u_0 after k steps from the current state, and dJ/d(sigma_a, sigma_s, q) per
        cell (FP64).  `out`: optional tuple of three float64 tensors/arrays to fill (host or CUDA);
        otherwise numpy arrays are returned.  The context then holds the state after k steps."""
        ptr, code, where, keep = _buf(w)
        if out is None:
            out = tuple(np.empty(self.shape, dtype=np.float64) for _ in range(3))
        bufs = [_buf(o) for o in out]
        for b in bufs:
            if b[1] != DTYPE_F64:
                raise TypeError("gradient buffers must be float64")
        ow = {b[2] for b in bufs}
        if len(ow) != 1:
            raise ValueError("gradient buffers must share the memory kind")
        J = _D()
        self._chk(lib().rtpn_adjoint(self._p, ptr, code, where, int(k), int(ckpt_every), bufs[0][0],
                                     bufs[1][0], bufs[2][0], ow.pop(), ctypes.byref(J)))
        return J.value, out

    def adjoint_release(self):
        """Free the work buffers the adjoint keeps on the device between calls."""
        self._chk(lib().rtpn_adjoint_release(self._p))

    def detector(self, w, out=None):
        """J = sum w u_0 on the current state (FP64, fixed order).  With `out` (a one-element float64
        CUDA tensor) J is written there without a host synchronisation and `out` is returned;
        otherwise J is returned as a Python float."""
        ptr, code, where, keep = _buf(w)
        if out is None:
            J = _D()
            self._chk(lib().rtpn_detector(self._p, ptr, code, where, ctypes.cast(ctypes.byref(J), _P), HOST))
            return J.value
        import torch

        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
            raise ValueError("out must be a CUDA float64 tensor with at least one element")
        self._chk(lib().rtpn_detector(self._p, ptr, code, where, _P(out.data_ptr()), DEVICE))
        return out

    def copy_planes_from(self, src: "Context", src_z: int, dst_z: int, nz: int, cls: int = -1):
        """Planes [src_z, src_z + nz) of class cls (-1: both) of src's state into planes
        [dst_z, dst_z + nz) of this context's (device to device, one strided copy)."""
        self._chk(lib().rtpn_copy_planes(self._p, int(dst_z), src._p, int(src_z), int(nz), int(cls)))

    def sum_u0(self) -> float:
        out = _D()
        self._chk(lib().rtpn_sum_u0(self._p, ctypes.byref(out)))
        return out.value

    def count_nonfinite(self) -> int:
        out = ctypes.c_longlong()
        rc = lib().rtpn_count_nonfinite(self._p, ctypes.byref(out))
        if rc not in (OK, ENONFINITE):
            self._chk(rc)
        return out.value

    def synchronize(self):
        self._chk(lib().rtpn_synchronize(self._p))


class _Instance(Context):
    """A batch member: the context is owned by the batch (never destroyed here)."""

    def __init__(self, ptr, N, shape, h, bc, precision):
        self._p = _P(ptr)
        self.N, self.shape, self.h, self.bc, self.precision = N, tuple(shape), h, bc, precision
        self.n_c = (N + 1) ** 2

    def close(self):
        self._p = None


class Batch:
    """Independent instances advanced together by one grouped launch per pass."""

    def __init__(self, instances, precision: str = "fp32"):
        """instances: iterable of (N, (nz, ny, nx), h, bc, dt or None)."""
        inst = list(instances)
        n = len(inst)
        arr_i = lambda vals: (_I * n)(*vals)
        arr_d = lambda vals: (_D * n)(*vals)
        Ns = arr_i([i[0] for i in inst])
        nz = arr_i([i[1][0] for i in inst])
        ny = arr_i([i[1][1] for i in inst])
        nx = arr_i([i[1][2] for i in inst])
        hs = arr_d([i[2] for i in inst])
        bcs = arr_i([BC[i[3]] for i in inst])
        dts = arr_d([float(i[4] or 0.0) for i in inst])
        p = _P()
        rc = lib().rtpn_batch_create(ctypes.byref(p), n, ctypes.cast(Ns, _P), ctypes.cast(nx, _P),
                                     ctypes.cast(ny, _P), ctypes.cast(nz, _P), ctypes.cast(hs, _P),
                                     ctypes.cast(bcs, _P), ctypes.cast(dts, _P), PRECISION[precision])
        if rc != OK:
            raise RtpnError(rc, lib().rtpn_last_error(None).decode() or lib().rtpn_strerror(rc).decode())
        self._p = p
        self.instances = [_Instance(lib().rtpn_batch_instance(p, i), inst[i][0], inst[i][1],
                                    inst[i][2], inst[i][3], precision) for i in range(n)]

    def _chk(self, rc):
        if rc != OK:
            raise RtpnError(rc, lib().rtpn_batch_last_error(self._p).decode() or
                            lib().rtpn_strerror(rc).decode())

    def __len__(self):
        return len(self.instances)

    def __getitem__(self, i) -> Context:
        return self.instances[i]

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._chk(lib().rtpn_batch_set_stream(self._p, _P(handle or 0)))

    def set_tile(self, tile):
        self._chk(lib().rtpn_batch_set_tile(self._p, *tile))

    def tile(self):
        t = [_I(), _I(), _I()]
        self._chk(lib().rtpn_batch_get_tile(self._p, *[ctypes.byref(v) for v in t]))
        return tuple(v.value for v in t)

    def step(self, k: int = 1):
        self._chk(lib().rtpn_batch_step(self._p, int(k)))

    def autotune(self, reps: int = 2):
        tile = (_I * 3)()
        ms = _D()
        self._chk(lib().rtpn_batch_autotune(self._p, int(reps), tile, ctypes.byref(ms)))
        return tuple(tile), ms.value

    def step_looped(self, k: int = 1):
        self._chk(lib().rtpn_batch_step_looped(self._p, int(k)))

    def synchronize(self):
        self._chk(lib().rtpn_batch_synchronize(self._p))

    def close(self):
        if getattr(self, "_p", None):
            for i in self.instances:
                i._p = None
            lib().rtpn_batch_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
