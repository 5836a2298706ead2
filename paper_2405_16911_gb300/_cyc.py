"""ctypes binding of libcyc (include/cyc.h): argument marshalling only.

Every entry point of the C ABI has a Python function of the same name.  Chunks and
outputs may be torch tensors (device or host), numpy arrays, or raw integer pointers.
All arithmetic happens in the CUDA library; if it is missing or no GPU is present,
``load()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcyc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cyc.h")

CYC_OK, CYC_EINVAL, CYC_ENOMEM, CYC_ECUDA, CYC_EAGAIN, CYC_ETIMEDOUT, CYC_ENODATA, CYC_ENOTSUP = \
    0, -1, -2, -3, -4, -5, -6, -7
CYC_CONV, CYC_CONJ, CYC_BOTH = 1, 2, 3
CYC_P_FP32, CYC_P_FP16, CYC_P_BF16X3 = 0, 1, 2
PRECISIONS = {"fp32": CYC_P_FP32, "fp16": CYC_P_FP16, "bf16x3": CYC_P_BF16X3}


class CycError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_strerror_py(code), code, msg))
        self.code = code


def _strerror_py(code):
    return {0: "success", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
            -4: "not admitted", -5: "timed out", -6: "no data", -7: "not supported"}.get(code, "error")


class cyc_params(ctypes.Structure):
    _fields_ = [("lags", ctypes.c_void_p), ("nlags", ctypes.c_int32),
                ("alphas", ctypes.c_void_p), ("nalphas", ctypes.c_int32),
                ("conj_flag", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n0", ctypes.c_int64), ("max_chunk", ctypes.c_int64),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int32)]


class cyc_server_params(ctypes.Structure):
    _fields_ = [("max_streams", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("mem_budget", ctypes.c_uint64), ("ring_samples", ctypes.c_int64),
                ("max_items", ctypes.c_int32), ("item_samples", ctypes.c_int64),
                ("device", ctypes.c_int32)]


class cyc_done(ctypes.Structure):
    _fields_ = [("sid", ctypes.c_int32), ("status", ctypes.c_int32), ("tag", ctypes.c_uint64),
                ("nsamples", ctypes.c_int64), ("submit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


_lib = None


def declared_functions(header: str = HEADER):
    """Names of the entry points declared in include/cyc.h."""
    with open(header) as f:
        return re.findall(r"CYC_API\s+[\w\s\*]+?\b(cyc_\w+)\s*\(", f.read())


def load(path: str = LIB_PATH):
    """Load libcyc.so (built in-tree by ``paper_2405_16911_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libcyc.so is not built (%s); run paper_2405_16911_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I32, I64, I = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    sig = {
        "cyc_create": ([P, I, P, I, I, P], I),
        "cyc_create_ex": ([P, P], I),
        "cyc_create_xy": ([P, P], I),
        "cyc_create_window": ([P, I64, I64, I64, I, P], I),
        "cyc_create_full": ([P, I32, I, P], I),
        "cyc_create_full_window": ([P, I32, I64, I64, I, P], I),
        "cyc_read_windows": ([P, P, I64, P, P], I),
        "cyc_read_spectrum": ([P, I32, I32, P], I),
        "cyc_detect": ([P, ctypes.c_double, I32, P, P, P], I),
        "cyc_set_wait_budget": ([P, I64], I),
        "cyc_sums": ([P, P, P, P], I),
        "cyc_set_n_eff": ([P, I64], I),
        "cyc_push": ([P, P, I64, I], I),
        "cyc_push_xy": ([P, P, P, I64, I], I),
        "cyc_read": ([P, P, P], I),
        "cyc_sync": ([P], I),
        "cyc_reset": ([P], I),
        "cyc_destroy": ([P], I),
        "cyc_save": ([P, P, P], I),
        "cyc_load": ([P, P, ctypes.c_size_t], I),
        "cyc_info": ([P, P, P, P, P], I),
        "cyc_phase_increment": ([ctypes.c_double, P], I),
        "cyc_estimate_static": ([P, I64, P, I, P, I, I, I64, P, P, P], I),
        "cyc_profile": ([P, I], I),
        "cyc_profile_read": ([P, P, P, P], I),
        "cyc_server_create": ([P, P], I),
        "cyc_server_destroy": ([P], I),
        "cyc_server_open": ([P, P, I, P, I, I, I64, P], I),
        "cyc_server_submit": ([P, I, P, I64, ctypes.c_uint64], I),
        "cyc_server_poll": ([P, P, I, P], I),
        "cyc_server_drain": ([P, ctypes.c_double], I),
        "cyc_server_read": ([P, I, P, P], I),
        "cyc_server_close": ([P, I], I),
        "cyc_server_stats": ([P, P, P, P, P], I),
        "cyc_net_create": ([P, ctypes.c_uint64, I, P], I),
        "cyc_net_destroy": ([P], I),
        "cyc_net_nparams": ([], I),
        "cyc_net_get_params": ([P, P], I),
        "cyc_net_set_params": ([P, P], I),
        "cyc_features": ([P, I64, I, P], I),
        "cyc_net_forward": ([P, P, I, P], I),
        "cyc_net_gradients": ([P, P, P, I, ctypes.c_float, P, P], I),
        "cyc_net_train_step": ([P, P, P, I, ctypes.c_float, ctypes.c_float, P], I),
        "cyc_propose": ([P, P, I64, I, I, ctypes.c_float, P, P, P, P], I),
        "cyc_strerror": ([I], ctypes.c_char_p),
        "cyc_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise CycError(rc, _lib.cyc_last_error().decode())
    return rc


def _ptr_info(obj):
    """(address, nbytes, on_device, keepalive) for a torch tensor, numpy array or int."""
    if isinstance(obj, int):
        return obj, None, None, None
    if isinstance(obj, np.ndarray):
        if not obj.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return obj.ctypes.data, obj.nbytes, 0, obj
    mod = type(obj).__module__
    if mod.startswith("torch"):
        if not obj.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return obj.data_ptr(), obj.numel() * obj.element_size(), 1 if obj.is_cuda else 0, obj
    raise TypeError("expected a torch tensor, numpy array or integer address, got %r" % type(obj))


# ----------------------------------------------------------------------------- entry points

def _nforms(conj_flag: int) -> int:
    return (1 if conj_flag & CYC_CONV else 0) + (1 if conj_flag & CYC_CONJ else 0)


def cyc_create(lags, alphas, conj_flag: int = CYC_BOTH) -> int:
    lib = load()
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    h = ctypes.c_void_p()
    _check(lib.cyc_create(lags.ctypes.data, lags.size, alphas.ctypes.data, alphas.size, conj_flag, ctypes.byref(h)))
    _shapes[h.value] = (_nforms(conj_flag), alphas.size, lags.size)
    return h.value


def cyc_create_ex(lags, alphas, conj_flag: int = CYC_BOTH, precision=CYC_P_FP32, n0: int = 0,
                  max_chunk: int = 0, cuda_stream: int = 0, device: int = 0, cross: bool = False,
                  window=None) -> int:
    """cross=True: cyc_create_xy, a stream with two inputs (cyc_push_xy); window=(win_len, hop,
    capacity): cyc_create_window (windowed output, cyc_read_windows)."""
    lib = load()
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    p = cyc_params(lags.ctypes.data, lags.size, alphas.ctypes.data, alphas.size, conj_flag, precision,
                   int(n0), int(max_chunk), cuda_stream or None, device)
    h = ctypes.c_void_p()
    if window is not None:
        wl, hp, cap = window
        _check(lib.cyc_create_window(ctypes.byref(p), int(wl), int(hp), int(cap), 1 if cross else 0, ctypes.byref(h)))
    else:
        _check((lib.cyc_create_xy if cross else lib.cyc_create_ex)(ctypes.byref(p), ctypes.byref(h)))
    _shapes[h.value] = (_nforms(conj_flag), alphas.size, lags.size)
    return h.value


def cyc_push(h: int, chunk, nsamples: int | None = None, on_device: int | None = None) -> None:
    addr, nbytes, dev, _keep = _ptr_info(chunk)
    if nsamples is None:
        if nbytes is None:
            raise ValueError("nsamples is required with a raw address")
        nsamples = nbytes // 8
    if on_device is None:
        if dev is None:
            raise ValueError("on_device is required with a raw address")
        on_device = dev
    _check(load().cyc_push(h, addr, int(nsamples), int(on_device)))


def cyc_create_xy(lags, alphas, conj_flag: int = CYC_BOTH, precision=CYC_P_FP32, n0: int = 0,
                  max_chunk: int = 0, cuda_stream: int = 0, device: int = 0) -> int:
    """A stream with two inputs x, y (the cross forms); feed it with cyc_push_xy."""
    return cyc_create_ex(lags, alphas, conj_flag, precision, n0, max_chunk, cuda_stream, device, cross=True)


def cyc_push_xy(h: int, x_chunk, y_chunk, nsamples: int | None = None, on_device: int | None = None) -> None:
    xa, xb, xd, _kx = _ptr_info(x_chunk)
    ya, yb, yd, _ky = _ptr_info(y_chunk)
    if nsamples is None:
        if xb is None or yb is None:
            raise ValueError("nsamples is required with raw addresses")
        if xb != yb:
            raise ValueError("x and y chunks differ in length")
        nsamples = xb // 8
    if on_device is None:
        if xd is None or xd != yd:
            raise ValueError("on_device is required with raw addresses or mixed host/device chunks")
        on_device = xd
    _check(load().cyc_push_xy(h, xa, ya, int(nsamples), int(on_device)))


def cyc_create_full(lags, A: int, conj_flag: int = CYC_BOTH, n0: int = 0, max_chunk: int = 0, cuda_stream: int = 0,
                    device: int = 0, cross: bool = False) -> int:
    """Full mode: every cycle frequency a_k = -1/2 + k/A (FP32 lag products folded mod A)."""
    lib = load()
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    p = cyc_params(lags.ctypes.data, lags.size, None, 0, conj_flag, CYC_P_FP32, int(n0), int(max_chunk),
                   cuda_stream or None, device)
    h = ctypes.c_void_p()
    _check(lib.cyc_create_full(ctypes.byref(p), int(A), 1 if cross else 0, ctypes.byref(h)))
    _shapes[h.value] = (_nforms(conj_flag), int(A), lags.size)
    return h.value


def cyc_create_full_window(lags, A: int, hop: int, capacity: int, conj_flag: int = CYC_BOTH, n0: int = 0,
                           max_chunk: int = 0, cuda_stream: int = 0, device: int = 0, cross: bool = False) -> int:
    """Full mode per window: every A samples' window (every hop) on the grid -1/2 + k/A."""
    lib = load()
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    p = cyc_params(lags.ctypes.data, lags.size, None, 0, conj_flag, CYC_P_FP32, int(n0), int(max_chunk),
                   cuda_stream or None, device)
    h = ctypes.c_void_p()
    _check(lib.cyc_create_full_window(ctypes.byref(p), int(A), int(hop), int(capacity), 1 if cross else 0,
                                      ctypes.byref(h)))
    _shapes[h.value] = (_nforms(conj_flag), int(A), lags.size)
    return h.value


def cyc_create_window(lags, alphas, win_len: int, hop: int, capacity: int, conj_flag: int = CYC_BOTH,
                      precision=CYC_P_FP32, n0: int = 0, max_chunk: int = 0, cuda_stream: int = 0, device: int = 0,
                      cross: bool = False) -> int:
    """A windowed stream: estimates over win_len reference samples every hop samples."""
    return cyc_create_ex(lags, alphas, conj_flag, precision, n0, max_chunk, cuda_stream, device, cross,
                         window=(win_len, hop, capacity))


def cyc_read_windows(h: int, max_win: int, out=None):
    """Completed windows, oldest first: (R [nwin][F][A][L] complex128 (a view of `out` or a new
    array), index k of the first window)."""
    F, A, L = cyc_shape(h)
    if out is None:
        out = np.empty((max_win, F, A, L), dtype=np.complex128)
    addr, nbytes, _dev, _keep = _ptr_info(out)
    if nbytes is not None and nbytes < max_win * F * A * L * 16:
        raise ValueError("output buffer too small")
    nw = ctypes.c_int64(0)
    k0 = ctypes.c_int64(0)
    _check(load().cyc_read_windows(h, addr, int(max_win), ctypes.byref(nw), ctypes.byref(k0)))
    return out[:nw.value], int(k0.value)


def cyc_read_spectrum(h: int, Q: int, taper: int = 0, out=None):
    """Cyclic spectra [F][A][Q] (complex128; `out` torch/numpy or a new numpy array)."""
    F, A, L = cyc_shape(h)
    if out is None:
        out = np.empty((F, A, int(Q)), dtype=np.complex128)
    addr, nbytes, _dev, _keep = _ptr_info(out)
    if nbytes is not None and nbytes < F * A * int(Q) * 16:
        raise ValueError("output buffer too small")
    _check(load().cyc_read_spectrum(h, int(Q), int(taper), addr))
    return out


def cyc_detect(h: int, kappa: float = 8.4, win: int = 16, flags=None, ratio=None):
    """Cycle-frequency detection on the stream's estimate: (flags [F][A] uint8 -- bit 0
    detected, bit 1 local maximum --, ratio [F][A] float32 or None, number detected).
    `flags` / `ratio` may be torch tensors or numpy arrays (host or device); by default new
    numpy arrays."""
    F, A, L = cyc_shape(h)
    if flags is None:
        flags = np.empty((F, A), dtype=np.uint8)
    if ratio is None:
        ratio = np.empty((F, A), dtype=np.float32)
    faddr, fn, _d1, _k1 = _ptr_info(flags)
    raddr, rn, _d2, _k2 = _ptr_info(ratio) if ratio is not False else (None, None, None, None)
    if (fn is not None and fn < F * A) or (rn is not None and rn < F * A * 4):
        raise ValueError("output buffer too small")
    nd = ctypes.c_int32(0)
    _check(load().cyc_detect(h, float(kappa), int(win), faddr, raddr, ctypes.byref(nd)))
    return flags, (None if ratio is False else ratio), int(nd.value)


def cyc_read(h: int, out=None):
    """Write R into `out` (torch/numpy, complex128 or float64 view) or return a new
    complex128 numpy array [F][A][L].  Returns (R, n_eff)."""
    lib = load()
    F, A, L = cyc_shape(h)
    neff = ctypes.c_int64(0)
    if out is None:
        out = np.empty((F, A, L), dtype=np.complex128)
    addr, nbytes, _dev, _keep = _ptr_info(out)
    if nbytes is not None and nbytes < F * A * L * 16:
        raise ValueError("output buffer too small")
    _check(lib.cyc_read(h, addr, ctypes.byref(neff)))
    return out, int(neff.value)


def cyc_sync(h: int) -> None:
    _check(load().cyc_sync(h))


def cyc_reset(h: int) -> None:
    _check(load().cyc_reset(h))


def cyc_destroy(h: int) -> None:
    if h:
        _shapes.pop(h, None)
        _check(load().cyc_destroy(h))


def cyc_save(h: int) -> bytes:
    lib = load()
    n = ctypes.c_size_t(0)
    _check(lib.cyc_save(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.cyc_save(h, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def cyc_load(h: int, blob: bytes) -> None:
    _check(load().cyc_load(h, blob, len(blob)))


def cyc_info(h: int):
    """(forms, unique cycle frequencies, samples pushed, N_eff)."""
    f, u = ctypes.c_int(0), ctypes.c_int(0)
    t, n = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().cyc_info(h, ctypes.byref(f), ctypes.byref(u), ctypes.byref(t), ctypes.byref(n)))
    return f.value, u.value, t.value, n.value


def cyc_estimate_static(x, T: int, lags, alphas, conj_flag: int, n0: int, out, cuda_stream: int = 0) -> int:
    """One-shot estimate with no allocation inside the library (see include/cyc.h).
    x, out: device tensors (or addresses) of the current device; returns N_eff.  The work
    is queued on `cuda_stream`; synchronise it before reading `out`."""
    lib = load()
    xa, _, _, _kx = _ptr_info(x)
    oa, _, _, _ko = _ptr_info(out)
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    neff = ctypes.c_int64(0)
    _check(lib.cyc_estimate_static(xa, int(T), lags.ctypes.data, lags.size, alphas.ctypes.data, alphas.size,
                                   int(conj_flag), int(n0), oa, ctypes.byref(neff), cuda_stream or None))
    return neff.value


def cyc_set_wait_budget(h: int, cycles: int) -> None:
    """SM cycles each bounded wait of the stream's tensor-core kernel waits (0: default)."""
    _check(load().cyc_set_wait_budget(h, int(cycles)))


class _DeviceArray:
    """A device buffer of the library, exposed to torch through __cuda_array_interface__."""

    def __init__(self, addr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (addr, False), "version": 3}


def cyc_sums(h: int):
    """(torch float64 tensor viewing the stream's device running sums, n_eff); adding into
    the tensor in place adds into the stream's sums (see include/cyc.h)."""
    import torch
    p = ctypes.c_void_p(0)
    nv = ctypes.c_int64(0)
    ne = ctypes.c_int64(0)
    _check(load().cyc_sums(h, ctypes.byref(p), ctypes.byref(nv), ctypes.byref(ne)))
    return torch.as_tensor(_DeviceArray(p.value, 2 * nv.value), device="cuda"), int(ne.value)


def cyc_set_n_eff(h: int, n_eff: int) -> None:
    _check(load().cyc_set_n_eff(h, int(n_eff)))


def cyc_phase_increment(a: float) -> int:
    """round(a * 2^64) mod 2^64: the u64 phase step the library uses for cycle frequency a."""
    v = ctypes.c_uint64(0)
    _check(load().cyc_phase_increment(float(a), ctypes.byref(v)))
    return v.value


def cyc_profile(h: int, enable: bool = True) -> None:
    _check(load().cyc_profile(h, int(bool(enable))))


def cyc_profile_read(h: int):
    """(projection ms, projection launches, all kernel launches) since the last call."""
    ms, pl, kl = ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().cyc_profile_read(h, ctypes.byref(ms), ctypes.byref(pl), ctypes.byref(kl)))
    return ms.value, pl.value, kl.value


def cyc_strerror(code: int) -> str:
    return load().cyc_strerror(code).decode()


def cyc_last_error() -> str:
    return load().cyc_last_error().decode()


# ----------------------------------------------------------------------------- serving

_srv_shapes: dict[tuple[int, int], tuple[int, int, int]] = {}


def cyc_server_create(max_streams: int = 256, precision="bf16x3", mem_budget: int = 0, ring_samples: int = 0,
                      max_items: int = 0, item_samples: int = 0, device: int = 0) -> int:
    lib = load()
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    p = cyc_server_params(max_streams, precision, mem_budget, ring_samples, max_items, item_samples, device)
    h = ctypes.c_void_p()
    _check(lib.cyc_server_create(ctypes.byref(p), ctypes.byref(h)))
    return h.value


def cyc_server_destroy(srv: int) -> None:
    if srv:
        for k in [k for k in _srv_shapes if k[0] == srv]:
            del _srv_shapes[k]
        _check(load().cyc_server_destroy(srv))


def cyc_server_open(srv: int, lags, alphas, conj_flag: int = CYC_BOTH, n0: int = 0) -> int:
    lib = load()
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    sid = ctypes.c_int(0)
    _check(lib.cyc_server_open(srv, lags.ctypes.data, lags.size, alphas.ctypes.data, alphas.size, conj_flag,
                               int(n0), ctypes.byref(sid)))
    _srv_shapes[(srv, sid.value)] = (_nforms(conj_flag), alphas.size, lags.size)
    return sid.value


def cyc_server_submit(srv: int, sid: int, chunk, nsamples: int | None = None, tag: int = 0) -> None:
    addr, nbytes, _dev, _keep = _ptr_info(chunk)
    if nsamples is None:
        if nbytes is None:
            raise ValueError("nsamples is required with a raw address")
        nsamples = nbytes // 8
    _check(load().cyc_server_submit(srv, sid, addr, int(nsamples), int(tag)))


def cyc_server_poll(srv: int, max_done: int = 4096):
    """Finished chunks as a list of (sid, status, tag, nsamples, submit_s, done_s)."""
    buf = (cyc_done * max_done)()
    n = ctypes.c_int(0)
    _check(load().cyc_server_poll(srv, buf, max_done, ctypes.byref(n)))
    return [(d.sid, d.status, d.tag, d.nsamples, d.submit_s, d.done_s) for d in buf[:n.value]]


def cyc_server_drain(srv: int, timeout_s: float = 60.0) -> None:
    _check(load().cyc_server_drain(srv, float(timeout_s)))


def cyc_server_read(srv: int, sid: int, out=None):
    F, A, L = _srv_shapes[(srv, sid)]
    if out is None:
        out = np.empty((F, A, L), dtype=np.complex128)
    addr, nbytes, _dev, _keep = _ptr_info(out)
    if nbytes is not None and nbytes < F * A * L * 16:
        raise ValueError("output buffer too small")
    neff = ctypes.c_int64(0)
    _check(load().cyc_server_read(srv, sid, addr, ctypes.byref(neff)))
    return out, int(neff.value)


def cyc_server_close(srv: int, sid: int) -> None:
    _srv_shapes.pop((srv, sid), None)
    _check(load().cyc_server_close(srv, sid))


def cyc_server_stats(srv: int):
    """(batches, items, busy ms, device bytes held by open streams)."""
    b, i = ctypes.c_int64(0), ctypes.c_int64(0)
    ms, by = ctypes.c_double(0), ctypes.c_uint64(0)
    _check(load().cyc_server_stats(srv, ctypes.byref(b), ctypes.byref(i), ctypes.byref(ms), ctypes.byref(by)))
    return b.value, i.value, ms.value, by.value


class Server:
    """Owning wrapper of a continuous-batching server."""

    def __init__(self, **kw):
        self.h = cyc_server_create(**kw)

    def open(self, lags, alphas, conj_flag: int = CYC_BOTH, n0: int = 0) -> int:
        return cyc_server_open(self.h, lags, alphas, conj_flag, n0)

    def submit(self, sid, chunk, nsamples=None, tag=0):
        cyc_server_submit(self.h, sid, chunk, nsamples, tag)

    def poll(self, max_done=4096):
        return cyc_server_poll(self.h, max_done)

    def drain(self, timeout_s=60.0):
        cyc_server_drain(self.h, timeout_s)

    def read(self, sid, out=None):
        return cyc_server_read(self.h, sid, out)

    def close_stream(self, sid):
        cyc_server_close(self.h, sid)

    def stats(self):
        return cyc_server_stats(self.h)

    def close(self):
        if self.h:
            cyc_server_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- proposer

def cyc_net_nparams() -> int:
    return int(load().cyc_net_nparams())


def cyc_net_create(params=None, seed: int = 0, device: int = 0) -> int:
    lib = load()
    h = ctypes.c_void_p()
    if params is not None:
        params = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if params.size != cyc_net_nparams():
            raise ValueError("expected %d parameters" % cyc_net_nparams())
    _check(lib.cyc_net_create(params.ctypes.data if params is not None else None, int(seed), device, ctypes.byref(h)))
    return h.value


def cyc_net_destroy(n: int) -> None:
    if n:
        _check(load().cyc_net_destroy(n))


def cyc_net_get_params(n: int) -> np.ndarray:
    out = np.empty(cyc_net_nparams(), dtype=np.float32)
    _check(load().cyc_net_get_params(n, out.ctypes.data))
    return out


def cyc_net_set_params(n: int, params) -> None:
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if params.size != cyc_net_nparams():
        raise ValueError("expected %d parameters" % cyc_net_nparams())
    _check(load().cyc_net_set_params(n, params.ctypes.data))


def cyc_features(x, T: int, nsig: int, feats) -> None:
    """x: device complex64 signals back to back (T samples each); feats: device FP16 [nsig][3][4096]."""
    xa, _, _, _k1 = _ptr_info(x)
    fa, _, _, _k2 = _ptr_info(feats)
    _check(load().cyc_features(xa, int(T), int(nsig), fa))


def cyc_net_forward(n: int, feats, B: int, logits) -> None:
    fa, _, _, _k1 = _ptr_info(feats)
    la, _, _, _k2 = _ptr_info(logits)
    _check(load().cyc_net_forward(n, fa, int(B), la))


def cyc_net_gradients(n: int, feats, labels, B: int, pos_weight: float = 1.0):
    """(gradients as a host float32 vector, loss)."""
    fa, _, _, _k1 = _ptr_info(feats)
    la, _, _, _k2 = _ptr_info(labels)
    g = np.empty(cyc_net_nparams(), dtype=np.float32)
    loss = ctypes.c_float(0)
    _check(load().cyc_net_gradients(n, fa, la, int(B), float(pos_weight), g.ctypes.data, ctypes.byref(loss)))
    return g, float(loss.value)


def cyc_net_train_step(n: int, feats, labels, B: int, lr: float, pos_weight: float = 1.0) -> float:
    fa, _, _, _k1 = _ptr_info(feats)
    la, _, _, _k2 = _ptr_info(labels)
    loss = ctypes.c_float(0)
    _check(load().cyc_net_train_step(n, fa, la, int(B), float(lr), float(pos_weight), ctypes.byref(loss)))
    return float(loss.value)


def cyc_propose(n: int, x, T: int | None = None, k: int = 32, tau: float = 0.9, on_device: int | None = None):
    """(alphas_conv[k], alphas_conj[k], confidence, used_fallback)."""
    xa, nb, dev, _k = _ptr_info(x)
    if T is None:
        T = nb // 8
    if on_device is None:
        on_device = dev
    ac = np.empty(k, dtype=np.float64)
    aj = np.empty(k, dtype=np.float64)
    conf = ctypes.c_float(0)
    fb = ctypes.c_int(0)
    _check(load().cyc_propose(n, xa, int(T), int(on_device), int(k), float(tau), ac.ctypes.data, aj.ctypes.data,
                              ctypes.byref(conf), ctypes.byref(fb)))
    return ac, aj, float(conf.value), bool(fb.value)


# shapes are tracked on the Python side for cyc_read's default output
_shapes: dict[int, tuple[int, int, int]] = {}


def cyc_shape(h: int):
    return _shapes[h]


class Stream:
    """Owning wrapper: ``with Stream(lags, alphas, ...) as s: s.push(x); R, n = s.read()``."""

    def __init__(self, lags, alphas, conj_flag: int = CYC_BOTH, precision=CYC_P_FP32, n0: int = 0,
                 max_chunk: int = 0, cuda_stream: int = 0, device: int = 0, cross: bool = False, window=None,
                 full: int = 0):
        """full=A: the uniform grid -1/2 + k/A by folding (alphas must be None); with
        window=(A, hop, capacity) as well, Full mode per window (cyc_create_full_window)."""
        if full:
            if alphas is not None:
                raise ValueError("full mode generates its own cycle frequencies; pass alphas=None")
            if window is not None:
                win_len, hop, capacity = window
                if win_len != full:
                    raise ValueError("a Full-mode window is A samples long")
                self.h = cyc_create_full_window(lags, full, hop, capacity, conj_flag, n0, max_chunk, cuda_stream,
                                                device, cross)
            else:
                self.h = cyc_create_full(lags, full, conj_flag, n0, max_chunk, cuda_stream, device, cross)
        else:
            self.h = cyc_create_ex(lags, alphas, conj_flag, precision, n0, max_chunk, cuda_stream, device, cross,
                                   window)
        self.shape = _shapes[self.h]
        self.cross = cross

    def push(self, chunk, nsamples=None, on_device=None, y=None):
        """One input: push(x); a cross stream: push(x, y=y)."""
        if self.cross:
            cyc_push_xy(self.h, chunk, y, nsamples, on_device)
        else:
            if y is not None:
                raise ValueError("this stream has one input")
            cyc_push(self.h, chunk, nsamples, on_device)

    def read(self, out=None):
        return cyc_read(self.h, out)

    def read_windows(self, max_win: int, out=None):
        return cyc_read_windows(self.h, max_win, out)

    def read_spectrum(self, Q: int, taper: int = 0, out=None):
        return cyc_read_spectrum(self.h, Q, taper, out)

    def detect(self, kappa: float = 8.4, win: int = 16, flags=None, ratio=None):
        return cyc_detect(self.h, kappa, win, flags, ratio)

    def set_wait_budget(self, cycles: int):
        cyc_set_wait_budget(self.h, cycles)

    def sums(self):
        return cyc_sums(self.h)

    def set_n_eff(self, n_eff: int):
        cyc_set_n_eff(self.h, n_eff)

    def sync(self):
        cyc_sync(self.h)

    def reset(self):
        cyc_reset(self.h)

    def save(self) -> bytes:
        return cyc_save(self.h)

    def load(self, blob: bytes):
        cyc_load(self.h, blob)

    def info(self):
        return cyc_info(self.h)

    def profile(self, enable: bool = True):
        cyc_profile(self.h, enable)

    def profile_read(self):
        return cyc_profile_read(self.h)

    def close(self):
        if self.h:
            cyc_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
