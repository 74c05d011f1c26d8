"""GB300-native online convolutional sparse coding (OCSC) -- Python binding.

A thin ctypes layer over ``libocsc.so`` (the C ABI declared in
``include/ocsc.h``).  Every step of the method runs in the library's CUDA
kernels; this module only marshals pointers, sizes and the CUDA stream.  There
is no CPU fallback: if the library is missing or no GPU is present, calls fail
loudly.

Low-level functions carry the C names (``ocsc_init``, ``ocsc_code``, ...);
:class:`OCSC` wraps them for torch CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libocsc.so")

STATUS = {
    0: "OCSC_OK", 1: "OCSC_EINVAL", 2: "OCSC_ENOMEM", 3: "OCSC_ECUDA", 4: "OCSC_ETIMEOUT",
    5: "OCSC_ESTATE", 6: "OCSC_EUNSUPPORTED", 7: "OCSC_ENUMERIC",
}


class OCSCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


MAX_FFT_SIZES = 12  # OCSC_MAX_FFT_SIZES


class ocsc_opts(ctypes.Structure):
    _fields_ = [
        ("Jz", ctypes.c_int), ("Jd", ctypes.c_int), ("pad", ctypes.c_int),
        ("max_batch", ctypes.c_int), ("fft_sizes", ctypes.c_int * MAX_FFT_SIZES), ("warm_start", ctypes.c_int),
        ("return_feasible", ctypes.c_int), ("rho_convention", ctypes.c_int),
        ("seed", ctypes.c_uint64), ("precision", ctypes.c_int), ("autotune", ctypes.c_int),
        ("graphs", ctypes.c_int), ("history", ctypes.c_int), ("persistent", ctypes.c_int),
        ("band_lo", ctypes.c_int), ("band_hi", ctypes.c_int),
    ]


class ocsc_tuning(ctypes.Structure):
    _fields_ = [("fold_threads", ctypes.c_int), ("spat_cb", ctypes.c_int), ("gram_sc", ctypes.c_int),
                ("plane_ctas", ctypes.c_int), ("plane_ahead", ctypes.c_int), ("plane_threads", ctypes.c_int)]


class ocsc_counters(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("samples_coded", ctypes.c_uint64),
                ("dict_updates", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64)]


class ocsc_server_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("check_every", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("mem_budget", ctypes.c_size_t), ("update_every", ctypes.c_int), ("learn", ctypes.c_int)]


class ocsc_served(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("iters", ctypes.c_int), ("primal", ctypes.c_double),
                ("dual", ctypes.c_double), ("dict_version", ctypes.c_uint64)]


KERNELS = ("image_spectrum", "code_resid", "code_plane", "fold_factor", "dstep", "vstep_cols",
           "vstep_project", "dict_norms", "vstep_spectrum", "history_tc", "persist")

_P = ctypes.c_void_p
_I = ctypes.c_int
_PROTOS = {
    "ocsc_default_opts": (None, [ctypes.POINTER(ocsc_opts)]),
    "ocsc_init": (_I, [ctypes.POINTER(_P), _I, _I, _I, ctypes.c_double, ctypes.c_double,
                       ctypes.POINTER(ocsc_opts), _P]),
    "ocsc_destroy": (None, [_P]),
    "ocsc_padded_size": (_I, [_P, _I, _I, ctypes.POINTER(_I)]),
    "ocsc_code": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I),
                       ctypes.POINTER(_P)]),
    "ocsc_update_dict": (_I, [_P]),
    "ocsc_get_dict": (_I, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "ocsc_set_dict": (_I, [_P, _P, _I]),
    "ocsc_sync": (_I, [_P]),
    "ocsc_last_error": (ctypes.c_char_p, [_P]),
    "ocsc_drop_pending": (_I, [_P]),
    "ocsc_get_state": (_I, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "ocsc_get_tuning": (_I, [_P, _I, _P]),
    "ocsc_set_tuning": (_I, [_P, _I, _P]),
    "ocsc_set_state": (_I, [_P, _P, ctypes.c_size_t]),
    "ocsc_objective": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double)]),
    "ocsc_objective_terms": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                  ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
    "ocsc_rel_diff": (_I, [_P, _P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)]),
    "ocsc_get_counters": (_I, [_P, ctypes.POINTER(ocsc_counters)]),
    "ocsc_profile": (_I, [_P, ctypes.c_uint]),
    "ocsc_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
    "ocsc_fft2_r2c": (_I, [_P, _I, _P, _P, _I]),
    "ocsc_fft2_c2r": (_I, [_P, _I, _P, _P, _I]),
    "ocsc_server_default_opts": (None, [ctypes.POINTER(ocsc_server_opts)]),
    "ocsc_server_create": (_I, [ctypes.POINTER(_P), _P, ctypes.POINTER(ocsc_server_opts)]),
    "ocsc_server_destroy": (None, [_P]),
    "ocsc_server_submit": (_I, [_P, ctypes.c_uint64, _P, _I, _I, _P]),
    "ocsc_server_step": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ocsc_server_poll": (_I, [_P, ctypes.POINTER(ocsc_served), _I, ctypes.POINTER(_I)]),
    "ocsc_psnr": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I),
                       ctypes.POINTER(_P), ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "ocsc_filter_order": (_I, [_P, ctypes.POINTER(_I)]),
    "ocsc_copy_dict": (_I, [_P, _P]),
    "ocsc_set_wait_limit": (_I, [_P, ctypes.c_uint64]),
    "ocsc_band_export": (_I, [_P, _I, _I, _P, _P]),
    "ocsc_band_fold": (_I, [_P, _I, _P, _P]),
    "ocsc_band_dict_step": (_I, [_P, _P]),
    "ocsc_band_project": (_I, [_P, _P, _I]),
    "ocsc_code_noalloc": (_I, [_P, _I, _I, _P, _I, _I, _I, ctypes.c_double, ctypes.c_double, _I, _P,
                               _P, ctypes.c_char_p, ctypes.c_size_t]),
}
EXPORTED = tuple(_PROTOS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libocsc.so (fails loudly if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, status: int):
    if status != 0:
        msg = lib().ocsc_last_error(ctx)
        raise OCSCError(status, msg.decode() if msg else "")


# --- low-level functions with the C names ------------------------------------

def ocsc_default_opts() -> ocsc_opts:
    o = ocsc_opts()
    lib().ocsc_default_opts(ctypes.byref(o))
    return o


def ocsc_init(K: int, filter_h: int, filter_w: int, lam: float, rho: float,
              opts: ocsc_opts | None = None, stream: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = lib().ocsc_init(ctypes.byref(ctx), K, filter_h, filter_w, lam, rho,
                         ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(stream))
    _check(None, st)
    return ctx


def ocsc_destroy(ctx) -> None:
    lib().ocsc_destroy(ctx)


def ocsc_padded_size(ctx, H: int, W: int) -> int:
    n = ctypes.c_int()
    _check(ctx, lib().ocsc_padded_size(ctx, H, W, ctypes.byref(n)))
    return n.value


def ocsc_code(ctx, x_ptrs, H, W, u_ptrs=None) -> None:
    n = len(x_ptrs)
    xs = (_P * n)(*x_ptrs)
    hs = (_I * n)(*H)
    ws = (_I * n)(*W)
    us = (_P * n)(*u_ptrs) if u_ptrs is not None else None
    _check(ctx, lib().ocsc_code(ctx, n, xs, hs, ws, us))


def ocsc_update_dict(ctx) -> None:
    _check(ctx, lib().ocsc_update_dict(ctx))


def ocsc_get_dict(ctx, D_host_ptr: int) -> int:
    v = ctypes.c_uint64()
    _check(ctx, lib().ocsc_get_dict(ctx, ctypes.c_void_p(D_host_ptr), ctypes.byref(v)))
    return v.value


def ocsc_set_dict(ctx, D_host_ptr: int, normalize: int) -> None:
    _check(ctx, lib().ocsc_set_dict(ctx, ctypes.c_void_p(D_host_ptr), normalize))


def ocsc_sync(ctx) -> None:
    _check(ctx, lib().ocsc_sync(ctx))


def ocsc_last_error(ctx) -> str:
    m = lib().ocsc_last_error(ctx)
    return m.decode() if m else ""


def ocsc_drop_pending(ctx) -> None:
    _check(ctx, lib().ocsc_drop_pending(ctx))


def ocsc_get_state(ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(ctx, lib().ocsc_get_state(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, lib().ocsc_get_state(ctx, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def ocsc_get_tuning(ctx, N: int) -> dict:
    t = ocsc_tuning()
    _check(ctx, lib().ocsc_get_tuning(ctx, N, ctypes.byref(t)))
    return {"fold_threads": t.fold_threads, "spat_cb": t.spat_cb, "gram_sc": t.gram_sc,
            "plane_ctas": t.plane_ctas, "plane_ahead": t.plane_ahead, "plane_threads": t.plane_threads}


def ocsc_set_tuning(ctx, N: int, **fields) -> None:
    t = ocsc_tuning()
    for k, v in fields.items():
        setattr(t, k, int(v))
    _check(ctx, lib().ocsc_set_tuning(ctx, N, ctypes.byref(t)))


def ocsc_set_state(ctx, state: bytes) -> None:
    buf = ctypes.create_string_buffer(state, len(state))
    _check(ctx, lib().ocsc_set_state(ctx, buf, len(state)))


def ocsc_objective(ctx, x_ptrs, H, W, u_ptrs):
    n = len(x_ptrs)
    out = (ctypes.c_double * n)()
    _check(ctx, lib().ocsc_objective(ctx, n, (_P * n)(*x_ptrs), (_I * n)(*H), (_I * n)(*W),
                                     (_P * n)(*u_ptrs), out))
    return list(out)


def ocsc_objective_terms(ctx, x_ptrs, H, W, u_ptrs):
    n = len(x_ptrs)
    r2 = (ctypes.c_double * n)()
    l1 = (ctypes.c_double * n)()
    _check(ctx, lib().ocsc_objective_terms(ctx, n, (_P * n)(*x_ptrs), (_I * n)(*H), (_I * n)(*W),
                                           (_P * n)(*u_ptrs), r2, l1))
    return list(r2), list(l1)


def ocsc_rel_diff(ctx, a_ptr: int, b_ptr: int, count: int) -> float:
    out = ctypes.c_double()
    _check(ctx, lib().ocsc_rel_diff(ctx, a_ptr, b_ptr, count, ctypes.byref(out)))
    return out.value


def ocsc_psnr(ctx, x_ptrs, H, W, u_ptrs, peak: float):
    n = len(x_ptrs)
    out = (ctypes.c_double * n)()
    _check(ctx, lib().ocsc_psnr(ctx, n, (_P * n)(*x_ptrs), (_I * n)(*H), (_I * n)(*W), (_P * n)(*u_ptrs),
                                peak, out))
    return list(out)


def ocsc_filter_order(ctx, K: int):
    out = (_I * K)()
    _check(ctx, lib().ocsc_filter_order(ctx, out))
    return list(out)


def ocsc_copy_dict(ctx, D_dev_ptr: int) -> None:
    _check(ctx, lib().ocsc_copy_dict(ctx, ctypes.c_void_p(D_dev_ptr)))


def ocsc_set_wait_limit(ctx, polls: int) -> None:
    _check(ctx, lib().ocsc_set_wait_limit(ctx, polls))


def ocsc_get_counters(ctx) -> ocsc_counters:
    c = ocsc_counters()
    _check(ctx, lib().ocsc_get_counters(ctx, ctypes.byref(c)))
    return c


def ocsc_profile(ctx, mask: int) -> None:
    _check(ctx, lib().ocsc_profile(ctx, mask))


def ocsc_profile_read(ctx, kernel: int):
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(ctx, lib().ocsc_profile_read(ctx, kernel, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def ocsc_fft2_r2c(ctx, N: int, x_ptr: int, X_ptr: int, planes: int) -> None:
    _check(ctx, lib().ocsc_fft2_r2c(ctx, N, ctypes.c_void_p(x_ptr), ctypes.c_void_p(X_ptr), planes))


def ocsc_fft2_c2r(ctx, N: int, X_ptr: int, x_ptr: int, planes: int) -> None:
    _check(ctx, lib().ocsc_fft2_c2r(ctx, N, ctypes.c_void_p(X_ptr), ctypes.c_void_p(x_ptr), planes))


NOALLOC_SCRATCH_BYTES = 32 << 20


def ocsc_code_noalloc(x_ptr: int, H: int, W: int, D_ptr: int, K: int, M: int, N: int, lam: float,
                      rho: float, Jz: int, u_ptr: int, stream: int = 0) -> None:
    """Code one image without any device allocation (see include/ocsc.h)."""
    buf = ctypes.create_string_buffer(512)
    st = lib().ocsc_code_noalloc(ctypes.c_void_p(x_ptr), H, W, ctypes.c_void_p(D_ptr), K, M, N, lam,
                                 rho, Jz, ctypes.c_void_p(u_ptr), ctypes.c_void_p(stream), buf, 512)
    if st != 0:
        raise OCSCError(st, buf.value.decode())


# --- torch convenience wrapper --------------------------------------------------

class OCSC:
    """One OCSC learner on the current CUDA device.

    Images and codes are torch CUDA float32 tensors; the dictionary is read and
    written as numpy float32 [K, M, M].  Work is queued on ``stream`` (default:
    torch's current stream when the object is created).
    """

    def __init__(self, K: int, M: int, lam: float, rho: float, *, stream=None, **opts):
        import torch

        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("OCSC needs a CUDA GPU; there is no CPU fallback")
        o = ocsc_default_opts()
        sizes = opts.pop("fft_sizes", None)
        if "fft_size" in opts:
            sizes = [opts.pop("fft_size")]
        if sizes is not None:
            if not 1 <= len(sizes) <= MAX_FFT_SIZES:
                raise ValueError(f"one to {MAX_FFT_SIZES} FFT sizes")
            o.fft_sizes = (ctypes.c_int * MAX_FFT_SIZES)(*(list(sizes) + [0] * (MAX_FFT_SIZES - len(sizes))))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = ocsc_init(K, M, M, lam, rho, o, self.stream.cuda_stream)
        self.sizes = [n for n in o.fft_sizes if n]
        self.K, self.M, self.N = K, M, self.sizes[0]
        self.opts = o

    def close(self):
        if getattr(self, "ctx", None):
            ocsc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def padded_size(self, H: int, W: int) -> int:
        return ocsc_padded_size(self.ctx, H, W)

    def code(self, images, out=None, want_codes: bool = True):
        """Code a list of 2D float32 CUDA tensors; returns [K, N, N] codes
        (N the padded size of each image)."""
        torch = self._torch
        xs = [im.contiguous() for im in images]
        for im in xs:
            if not (im.is_cuda and im.dtype == torch.float32 and im.dim() == 2):
                raise ValueError("images must be 2D float32 CUDA tensors")
        if out is None and want_codes:
            out = []
            for im in xs:
                n = self.padded_size(im.shape[0], im.shape[1])
                out.append(torch.empty((self.K, n, n), device=im.device, dtype=torch.float32))
        ocsc_code(self.ctx, [im.data_ptr() for im in xs], [im.shape[0] for im in xs],
                  [im.shape[1] for im in xs], [u.data_ptr() for u in out] if out is not None else None)
        self._keep = xs  # images must outlive the queued work
        return out

    def update_dict(self):
        ocsc_update_dict(self.ctx)

    def get_dict(self):
        import numpy as np

        D = np.empty((self.K, self.M, self.M), np.float32)
        self.version = ocsc_get_dict(self.ctx, D.ctypes.data)
        return D

    def set_dict(self, D, normalize: bool = True):
        import numpy as np

        D = np.ascontiguousarray(D, dtype=np.float32)
        if D.shape != (self.K, self.M, self.M):
            raise ValueError(f"dictionary must be {(self.K, self.M, self.M)}")
        ocsc_set_dict(self.ctx, D.ctypes.data, int(normalize))

    def sync(self):
        ocsc_sync(self.ctx)

    def drop_pending(self):
        ocsc_drop_pending(self.ctx)

    def get_state(self) -> bytes:
        """Checkpoint of the learner (no samples may be pending)."""
        return ocsc_get_state(self.ctx)

    def set_tuning(self, N: int, **fields) -> None:
        """Pin tile shapes of FFT size N (ocsc_set_tuning); fields as tuning()."""
        ocsc_set_tuning(self.ctx, N, **fields)

    def tuning(self, N: int) -> dict:
        """Tile shapes the autotuner picked for FFT size N."""
        return ocsc_get_tuning(self.ctx, N)

    def set_state(self, state: bytes) -> None:
        """Load a checkpoint saved by a learner of the same shape and parameters."""
        ocsc_set_state(self.ctx, state)

    def objective(self, images, codes):
        """Per-sample objective of eq. (ocsc0) against the current dictionary."""
        xs = [im.contiguous() for im in images]
        us = [u.contiguous() for u in codes]
        return ocsc_objective(self.ctx, [im.data_ptr() for im in xs], [im.shape[0] for im in xs],
                              [im.shape[1] for im in xs], [u.data_ptr() for u in us])

    def objective_terms(self, images, codes):
        """(||x - sum_k D_k (*) U_k||^2, ||U||_1) per sample, padded domain."""
        xs = [im.contiguous() for im in images]
        us = [u.contiguous() for u in codes]
        return ocsc_objective_terms(self.ctx, [im.data_ptr() for im in xs], [im.shape[0] for im in xs],
                                    [im.shape[1] for im in xs], [u.data_ptr() for u in us])

    def psnr(self, images, codes, peak: float = 255.0):
        """Per-sample 10 log10(peak^2 P / ||x_rec - x||^2) over the padded
        P = N x N domain (Sec. IV; the paper uses peak 255 for 8-bit images)."""
        xs = [im.contiguous() for im in images]
        us = [u.contiguous() for u in codes]
        return ocsc_psnr(self.ctx, [im.data_ptr() for im in xs], [im.shape[0] for im in xs],
                         [im.shape[1] for im in xs], [u.data_ptr() for u in us], float(peak))

    def filter_order(self):
        """Filter indices in ascending order of their sample variance (Sec. IV)."""
        import numpy as np

        return np.asarray(ocsc_filter_order(self.ctx, self.K), np.int64)

    def dict_device(self, out=None):
        """The filters D_t as a [K, M, M] float32 CUDA tensor (device copy)."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.K, self.M, self.M), device="cuda", dtype=torch.float32)
        ocsc_copy_dict(self.ctx, out.data_ptr())
        return out

    # --- frequency-band sharding of the dictionary step (see bands.py) ---------

    def band_rows(self):
        """(k1_lo, k1_hi) of this band context."""
        return self.opts.band_lo, self.opts.band_hi

    def band_export(self, k1_lo: int, k1_hi: int, n: int):
        """The n pending samples' Z~ and x~ rows k1 in [k1_lo, k1_hi) as complex64
        CUDA tensors [n, K, rows * (N/2+1)] and [n, rows * (N/2+1)]."""
        torch = self._torch
        fb = (k1_hi - k1_lo) * (self.N // 2 + 1)
        Z = torch.empty((n, self.K, fb), device="cuda", dtype=torch.complex64)
        x = torch.empty((n, fb), device="cuda", dtype=torch.complex64)
        _check(self.ctx, lib().ocsc_band_export(self.ctx, k1_lo, k1_hi, ctypes.c_void_p(Z.data_ptr()),
                                                ctypes.c_void_p(x.data_ptr())))
        return Z, x

    def band_fold(self, Z, x):
        """Fold a mini-batch's band rows (global sample order) and factor the band."""
        Z = Z.contiguous()
        x = x.contiguous()
        self._keep_band = (Z, x)
        _check(self.ctx, lib().ocsc_band_fold(self.ctx, Z.shape[0], ctypes.c_void_p(Z.data_ptr()),
                                              ctypes.c_void_p(x.data_ptr())))

    def band_dict_step(self, out=None):
        """The band's share of the support sums alpha [K, M, M] (float32 CUDA)."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.K, self.M, self.M), device="cuda", dtype=torch.float32)
        _check(self.ctx, lib().ocsc_band_dict_step(self.ctx, ctypes.c_void_p(out.data_ptr())))
        return out

    def band_project(self, alpha, last: bool):
        alpha = alpha.contiguous()
        self._keep_alpha = alpha
        _check(self.ctx, lib().ocsc_band_project(self.ctx, ctypes.c_void_p(alpha.data_ptr()), int(last)))

    def set_wait_limit(self, polls: int):
        """Poll budget of the bounded device waits (failure-path tests)."""
        ocsc_set_wait_limit(self.ctx, int(polls))

    def rel_diff(self, a, b) -> float:
        """||a - b|| / ||a|| of two float32 CUDA tensors of the same size."""
        a = a.contiguous()
        b = b.contiguous()
        if a.numel() != b.numel():
            raise ValueError("sizes differ")
        return ocsc_rel_diff(self.ctx, a.data_ptr(), b.data_ptr(), a.numel())

    def fit(self, images, max_passes: int = 10, tol: float = 1e-3, batch: int = 1):
        """Online passes over `images` (Algorithm 3 per mini-batch) until the
        stopping rule of Sec. IV holds: the relative change of the codes of the
        current mini-batch against the previous pass and of the dictionary
        against the previous update both below tol (both relative changes are
        taken on the device, ocsc_rel_diff).  Returns a dict with the pass and
        step where it stopped (or max_passes) and the last changes."""

        prev = [None] * len(images)
        D_old = self.dict_device()
        D_new = self.dict_device()
        last = {"code_change": float("inf"), "dict_change": float("inf")}
        for p in range(max_passes):
            for t in range(0, len(images), batch):
                idx = list(range(t, min(t + batch, len(images))))
                us = self.code([images[i] for i in idx])
                self.update_dict()
                self.dict_device(out=D_new)
                dz = max(self.rel_diff(u, prev[i]) if prev[i] is not None else float("inf")
                         for u, i in zip(us, idx))
                dd = self.rel_diff(D_new, D_old)
                for u, i in zip(us, idx):
                    prev[i] = u
                D_old, D_new = D_new, D_old
                last = {"code_change": dz, "dict_change": dd}
                if dz < tol and dd < tol:
                    return {"stopped": True, "pass": p, "step": t // batch, **last}
        return {"stopped": False, "pass": max_passes, "step": None, **last}

    def counters(self) -> dict:
        c = ocsc_get_counters(self.ctx)
        return {"kernel_launches": c.kernel_launches, "samples_coded": c.samples_coded,
                "dict_updates": c.dict_updates, "graph_launches": c.graph_launches}

    def profile(self, kernels=KERNELS):
        """Time every launch of the named kernel classes with CUDA events."""
        mask = 0
        for k in kernels:
            mask |= 1 << KERNELS.index(k)
        ocsc_profile(self.ctx, mask)

    def profile_read(self, kernels=KERNELS) -> dict:
        """{kernel: (total ms, launches)} since the last read (synchronises)."""
        return {k: ocsc_profile_read(self.ctx, KERNELS.index(k)) for k in kernels}

    def fft2_r2c(self, x):
        torch = self._torch
        x = x.contiguous()
        N = x.shape[-1]
        X = torch.empty((x.shape[0], N, N // 2 + 1), device=x.device, dtype=torch.complex64)
        ocsc_fft2_r2c(self.ctx, N, x.data_ptr(), X.data_ptr(), x.shape[0])
        return X

    def fft2_c2r(self, X):
        torch = self._torch
        X = X.contiguous()
        N = X.shape[-2]
        x = torch.empty((X.shape[0], N, N), device=X.device, dtype=torch.float32)
        ocsc_fft2_c2r(self.ctx, N, X.data_ptr(), x.data_ptr(), X.shape[0])
        return x


class Server:
    """Continuous-batching request server over an :class:`OCSC` learner.

    ``submit`` queues an image (2D float32 CUDA tensor) and returns the output
    tensor that will hold its code; ``step`` runs one scheduling round; ``poll``
    returns the completed requests as dicts.  Output tensors and images are
    kept alive here until their request completes.
    """

    def __init__(self, learner: "OCSC", **opts):
        self.learner = learner
        o = ocsc_server_opts()
        lib().ocsc_server_default_opts(ctypes.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown server option {k}")
            setattr(o, k, v)
        h = ctypes.c_void_p()
        _check(learner.ctx, lib().ocsc_server_create(ctypes.byref(h), learner.ctx, ctypes.byref(o)))
        self.h = h
        self.opts = o
        self._live = {}

    def close(self):
        if getattr(self, "h", None):
            lib().ocsc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, rid: int, image, out=None):
        torch = self.learner._torch
        x = image.contiguous()
        n = self.learner.padded_size(x.shape[0], x.shape[1])
        if out is None:
            out = torch.empty((self.learner.K, n, n), device=x.device, dtype=torch.float32)
        _check(self.learner.ctx, lib().ocsc_server_submit(self.h, rid, ctypes.c_void_p(x.data_ptr()),
                                                          x.shape[0], x.shape[1],
                                                          ctypes.c_void_p(out.data_ptr())))
        self._live[rid] = (x, out)
        return out

    def step(self):
        a, q = _I(), _I()
        _check(self.learner.ctx, lib().ocsc_server_step(self.h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, max_items: int = 4096):
        buf = (ocsc_served * max_items)()
        n = _I()
        _check(self.learner.ctx, lib().ocsc_server_poll(self.h, buf, max_items, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            d = buf[i]
            x, u = self._live.pop(d.id, (None, None))
            out.append({"id": d.id, "iters": d.iters, "primal": d.primal, "dual": d.dual,
                        "dict_version": d.dict_version, "code": u})
        return out

