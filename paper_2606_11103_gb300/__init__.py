"""GB300-native heterogeneous power-law attenuation FDTD (Python binding).

The computation lives in ``libfullwave_gb.so`` (hand-written sm_103a CUDA and
host C++).  This module only marshals arguments into the C ABI declared in
``include/fullwave_gb.h``: the raw functions keep the C names (``fw_*``), and
``Medium`` / ``fit_relaxation`` are small conveniences over them.  PyTorch is
used only for device memory (an optional allocator hook) and streams.  There
is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    FW_ERR_ARG, FW_ERR_CUDA, FW_ERR_NOMEM, FW_ERR_STATE, FW_ERR_UNSTABLE, FW_ERR_UNSUPPORTED, FW_OK,
    FW_FIELD_P, FW_FIELD_PSI1, FW_FIELD_PSI1P, FW_FIELD_PSI2, FW_FIELD_PSI2P, FW_FIELD_V,
    FW_STORE_BF16, FW_STORE_F16, FW_STORE_F32, FW_STORE_F64, FwError, check, fw_fit_opts, fw_fit_report,
    fw_grid, fw_medium_info, fw_relax_params,
)

STORAGE = {"f32": FW_STORE_F32, "bf16": FW_STORE_BF16, "f16": FW_STORE_F16, "f64": FW_STORE_F64}


def lib():
    return _lib.load()


def __getattr__(name):
    # raw C entry points under their C names: paper_2606_11103_gb300.fw_run(...)
    if name.startswith("fw_") and name in _lib.SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


# ---------------------------------------------------------------------------
# marshalling helpers


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class _Buf:
    """A contiguous buffer of a given dtype: numpy (host) or torch (host/device)."""

    def __init__(self, a, dtype):
        self.keep = None
        try:
            import torch
            if isinstance(a, torch.Tensor):
                want = {np.float32: torch.float32, np.float64: torch.float64, np.uint8: torch.uint8,
                        np.int32: torch.int32}.get(dtype)
                if want is None and a.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
                    want = a.dtype          # 16-bit class indices are passed bit for bit
                if want is not None:
                    t = a.detach().to(want).contiguous()
                    self.keep = t
                    self.ptr = C.c_void_p(t.data_ptr())
                    return
                a = a.detach().cpu().numpy()
        except ImportError:  # pragma: no cover
            pass
        arr = np.ascontiguousarray(a, dtype=dtype)
        self.keep = arr
        self.ptr = C.c_void_p(arr.ctypes.data)


def make_grid(shape, dx, dt=0.0, cfl=0.0, pml=0, transition=0, f0=3e6, pml_r0=0.0, layer_relax=False,
              time_order=2) -> fw_grid:
    """fw_grid from a numpy-order shape (ny, nx) or (nz, ny, nx).  layer_relax:
    keep the caller's relaxation classes inside the absorbing layer instead of
    inheriting the nearest interior class.  time_order: 2 (leapfrog) or 4
    (the time-space stencil)."""
    g = fw_grid()
    g.ndim = len(shape)
    if g.ndim == 2:
        g.ny, g.nx, g.nz = int(shape[0]), int(shape[1]), 1
    elif g.ndim == 3:
        g.nz, g.ny, g.nx = (int(s) for s in shape)
    else:
        raise ValueError("shape must be 2D or 3D")
    g.dx, g.dt, g.cfl = float(dx), float(dt), float(cfl)
    g.pml, g.transition = int(pml), int(transition)
    g.f0, g.pml_r0 = float(f0), float(pml_r0)
    g.layer_relax = int(bool(layer_relax))
    g.time_order = int(time_order)
    return g


def relax_params(kappa1, kappa2, d1, alpha1, d2, alpha2) -> fw_relax_params:
    p = fw_relax_params()
    n = len(d1)
    p.n_mech = n
    p.kappa1, p.kappa2 = float(kappa1), float(kappa2)
    for i in range(n):
        p.d1[i], p.alpha1[i] = float(d1[i]), float(alpha1[i])
        p.d2[i], p.alpha2[i] = float(d2[i]), float(alpha2[i])
    return p


def fit_opts(**kw) -> fw_fit_opts:
    o = fw_fit_opts()
    lib().fw_fit_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "w":
            o.n_w = len(v)
            for i, x in enumerate(v):
                o.w[i] = float(x)
        else:
            setattr(o, k, v)
    return o


def fit_relaxation(alpha0, y, n_mech=2, **opts):
    """fw_fit_relaxation: returns (fw_relax_params, fw_fit_report)."""
    p, r = fw_relax_params(), fw_fit_report()
    o = fit_opts(**opts)
    check(lib().fw_fit_relaxation(float(alpha0), float(y), int(n_mech), C.byref(o), C.byref(p), C.byref(r)),
          "fw_fit_relaxation")
    return p, r


def model_wavenumber(p: fw_relax_params, c, f_hz):
    f = np.ascontiguousarray(f_hz, dtype=np.float64)
    kr, ki = np.empty_like(f), np.empty_like(f)
    D = C.POINTER(C.c_double)
    check(lib().fw_model_wavenumber(C.byref(p), float(c), f.ctypes.data_as(D), f.size,
                                    kr.ctypes.data_as(D), ki.ctypes.data_as(D)), "fw_model_wavenumber")
    return kr + 1j * ki


_alloc_refs = []


def use_torch_allocator(enable: bool = True):
    """Route every later medium's device memory through torch's caching allocator."""
    if not enable:
        lib().fw_set_allocator(_lib.ALLOCFN(), _lib.FREEFN(), None)
        return
    import torch

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:  # noqa: BLE001
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = _lib.ALLOCFN(_alloc), _lib.FREEFN(_free)
    _alloc_refs[:] = [fa, ff]
    lib().fw_set_allocator(fa, ff, None)


# ---------------------------------------------------------------------------
# medium


class Medium:
    """Owner of one ``fw_medium*`` (device-resident state and maps)."""

    def __init__(self, handle, shape):
        self.h = handle
        self.shape = tuple(shape)

    # -- construction ---------------------------------------------------------
    @classmethod
    def from_classes(cls, shape, dx, c, rho, class_idx, classes, dt=0.0, cfl=0.0, beta=None, pml=0,
                     transition=0, f0=3e6, storage="f32", stream=None, layer_relax=False, time_order=2):
        g = make_grid(shape, dx, dt, cfl, pml, transition, f0, layer_relax=layer_relax, time_order=time_order)
        arr = (fw_relax_params * len(classes))(*classes)
        bc, br = _Buf(c, np.float32), _Buf(rho, np.float32)
        bb = _Buf(beta, np.float32) if beta is not None else None
        bk = _Buf(class_idx, np.uint16)
        h = C.c_void_p()
        check(lib().fw_create_medium_classes(C.byref(g), bc.ptr, br.ptr, bb.ptr if bb else None, bk.ptr,
                                             arr, len(classes), STORAGE.get(storage, storage), _stream(stream),
                                             C.byref(h)), "fw_create_medium_classes")
        return cls(h, shape)

    @classmethod
    def from_maps(cls, shape, dx, c, rho, alpha0, y, n_mech=2, dt=0.0, cfl=0.0, beta=None, pml=0,
                  transition=0, f0=3e6, storage="f32", stream=None, layer_relax=False, time_order=2, **fit_kw):
        g = make_grid(shape, dx, dt, cfl, pml, transition, f0, layer_relax=layer_relax, time_order=time_order)
        o = fit_opts(**fit_kw)
        if "c0" not in fit_kw:
            o.c0 = 0.0           # per-class mean sound speed
        bufs = [_Buf(a, np.float32) for a in (c, rho, alpha0, y)]
        bb = _Buf(beta, np.float32) if beta is not None else None
        h = C.c_void_p()
        check(lib().fw_create_medium(C.byref(g), bufs[0].ptr, bufs[1].ptr, bb.ptr if bb else None, bufs[2].ptr,
                                     bufs[3].ptr, int(n_mech), STORAGE.get(storage, storage), C.byref(o),
                                     _stream(stream), C.byref(h)), "fw_create_medium")
        return cls(h, shape)

    # -- sources / receivers --------------------------------------------------
    def set_sources(self, mask, waves, wave_of=None):
        w = np.ascontiguousarray(np.atleast_2d(waves), dtype=np.float32)
        bm = _Buf(mask, np.uint8)
        bo = _Buf(wave_of, np.int32) if wave_of is not None else None
        check(lib().fw_set_sources(self.h, bm.ptr, C.c_void_p(w.ctypes.data), w.shape[0], w.shape[1],
                                   bo.ptr if bo else None), "fw_set_sources")

    def set_receivers(self, mask, n_steps, decim=1):
        bm = _Buf(mask, np.uint8)
        check(lib().fw_set_receivers(self.h, bm.ptr, int(decim), int(n_steps)), "fw_set_receivers")

    # -- stepping ---------------------------------------------------------------
    def step(self, n, stream=None):
        check(lib().fw_step(self.h, int(n), _stream(stream)), "fw_step")

    def run(self, n, stream=None):
        check(lib().fw_run(self.h, int(n), _stream(stream)), "fw_run")

    # -- I/O ----------------------------------------------------------------------
    def read_field(self, which=FW_FIELD_P, idx=0, f64=False, out=None, stream=None):
        dt = np.float64 if f64 else np.float32
        if out is None:
            out = np.empty(self.shape, dtype=dt)
        ptr = C.c_void_p(out.data_ptr()) if hasattr(out, "data_ptr") else C.c_void_p(out.ctypes.data)
        check(lib().fw_read_field(self.h, int(which), int(idx), ptr, int(bool(f64)), _stream(stream)),
              "fw_read_field")
        return out

    def write_field(self, which, idx, values, f64=False, stream=None):
        b = _Buf(values, np.float64 if f64 else np.float32)
        check(lib().fw_write_field(self.h, int(which), int(idx), b.ptr, int(bool(f64)), _stream(stream)),
              "fw_write_field")

    def receivers(self, f64=False, out=None, stream=None):
        inf = self.info()
        dt = np.float64 if f64 else np.float32
        if out is None:
            out = np.zeros((inf["n_rcv"], inf["n_rec"]), dtype=dt)
        ptr = C.c_void_p(out.data_ptr()) if hasattr(out, "data_ptr") else C.c_void_p(out.ctypes.data)
        check(lib().fw_read_receivers(self.h, ptr, int(bool(f64)), _stream(stream)), "fw_read_receivers")
        return out

    def gradient(self, n_steps, G, alpha0=None, checkpoint=0, f64=False, out=None, stream=None):
        """fw_gradient: run n_steps forward (as run()) and return (dL/dc,
        dL/dalpha0) of L = sum G * traces on the user grid.  G [n_rcv, n_rec];
        alpha0 the medium's alpha0 map, or None for dL/ds.  Host (numpy) or
        device (torch) buffers; ``out`` = (grad_c, grad_alpha0) to fill."""
        dt = np.float64 if f64 else np.float32
        bG = _Buf(G, dt)
        ba = _Buf(alpha0, dt) if alpha0 is not None else None
        if out is None:
            out = (np.empty(self.shape, dt), np.empty(self.shape, dt))
        ptrs = [C.c_void_p(o.data_ptr()) if hasattr(o, "data_ptr") else C.c_void_p(o.ctypes.data) for o in out]
        check(lib().fw_gradient(self.h, int(n_steps), int(checkpoint), bG.ptr, ba.ptr if ba else None,
                                ptrs[0], ptrs[1], int(bool(f64)), _stream(stream)), "fw_gradient")
        return out

    def state_bytes(self):
        n = C.c_size_t()
        check(lib().fw_state_bytes(self.h, C.byref(n)), "fw_state_bytes")
        return n.value

    def save_state(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.state_bytes(), dtype=np.uint8)
        ptr = C.c_void_p(out.data_ptr()) if hasattr(out, "data_ptr") else C.c_void_p(out.ctypes.data)
        check(lib().fw_save_state(self.h, ptr, _stream(stream)), "fw_save_state")
        return out

    def load_state(self, buf, stream=None):
        ptr = C.c_void_p(buf.data_ptr()) if hasattr(buf, "data_ptr") else C.c_void_p(np.ascontiguousarray(buf).ctypes.data)
        check(lib().fw_load_state(self.h, ptr, _stream(stream)), "fw_load_state")

    def status(self):
        m = C.c_float()
        rc = lib().fw_status(self.h, C.byref(m))
        return rc, m.value

    def info(self):
        i = fw_medium_info()
        check(lib().fw_medium_get_info(self.h, C.byref(i)), "fw_medium_get_info")
        return {k: getattr(i, k) for k, _ in fw_medium_info._fields_}

    def close(self):
        if self.h:
            lib().fw_destroy_medium(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


# ---------------------------------------------------------------------------
# serving


class Server:
    """Owner of one ``fw_server*`` (continuous batching of simulation
    requests on the current device).  ``submit`` keeps the request's buffers
    alive until its completion has been polled."""

    def __init__(self, hbm_budget, max_active=8, chunk_steps=32, n_streams=8, policy=0, short_work=0.0):
        o = _lib.fw_server_opts()
        o.hbm_budget, o.max_active, o.chunk_steps, o.n_streams = int(hbm_budget), int(max_active), \
            int(chunk_steps), int(n_streams)
        o.policy, o.short_work = int(policy), float(short_work)
        self.h = C.c_void_p()
        check(lib().fw_server_create(C.byref(o), C.byref(self.h)), "fw_server_create")
        self._keep = {}

    def submit(self, shape, dx, dt, c, rho, class_idx, classes, n_steps, src_mask=None, waves=None, wave_of=None,
               rcv_mask=None, decim=1, beta=None, pml=0, transition=0, f0=3e6, storage="f32", traces_out=None,
               tag=0, time_order=2):
        """Queue one request; returns (id, traces_out).  traces_out (numpy or
        torch, float32 [n_rcv, n_rec]) is filled at completion."""
        r = _lib.fw_request()
        r.grid = make_grid(shape, dx, dt, 0.0, pml, transition, f0, time_order=time_order)
        keep = [_Buf(c, np.float32), _Buf(rho, np.float32), _Buf(class_idx, np.uint16)]
        r.c, r.rho, r.class_idx = keep[0].ptr, keep[1].ptr, keep[2].ptr
        if beta is not None:
            keep.append(_Buf(beta, np.float32))
            r.beta = keep[-1].ptr
        arr = (fw_relax_params * len(classes))(*classes)
        keep.append(arr)
        r.classes, r.n_classes = arr, len(classes)
        r.storage = STORAGE.get(storage, storage)
        n_rcv = 0
        if src_mask is not None:
            w = np.ascontiguousarray(np.atleast_2d(waves), dtype=np.float32)
            keep += [_Buf(src_mask, np.uint8), w]
            r.src_mask, r.waveforms, r.n_wave = keep[-2].ptr, C.c_void_p(w.ctypes.data), w.shape[0]
            if wave_of is not None:
                keep.append(_Buf(wave_of, np.int32))
                r.wave_of = keep[-1].ptr
        if rcv_mask is not None:
            keep.append(_Buf(rcv_mask, np.uint8))
            r.rcv_mask = keep[-1].ptr
            n_rcv = int(np.count_nonzero(np.asarray(rcv_mask.cpu() if hasattr(rcv_mask, "cpu") else rcv_mask)))
        r.decim, r.n_steps, r.tag = int(decim), int(n_steps), int(tag)
        if traces_out is None and n_rcv:
            traces_out = np.zeros((n_rcv, (n_steps + decim - 1) // decim), np.float32)
        if traces_out is not None:
            r.traces_out = C.c_void_p(traces_out.data_ptr() if hasattr(traces_out, "data_ptr")
                                      else traces_out.ctypes.data)
        rid = C.c_longlong()
        check(lib().fw_server_submit(self.h, C.byref(r), C.byref(rid)), "fw_server_submit")
        self._keep[rid.value] = (r, keep, traces_out)
        return rid.value, traces_out

    def poll(self, timeout=0.0, max_n=256):
        """Completed requests as dicts (each returned once)."""
        out = (_lib.fw_completion * max_n)()
        n = C.c_int()
        check(lib().fw_server_poll(self.h, out, max_n, C.byref(n), float(timeout)), "fw_server_poll")
        res = []
        for k in range(n.value):
            d = {f: getattr(out[k], f) for f, _ in _lib.fw_completion._fields_}
            d["traces"] = self._keep.pop(d["id"], (None, None, None))[2]
            res.append(d)
        return res

    def cancel(self, rid):
        check(lib().fw_server_cancel(self.h, C.c_longlong(rid)), "fw_server_cancel")

    def stats(self):
        st = _lib.fw_server_stats()
        check(lib().fw_server_stats_get(self.h, C.byref(st)), "fw_server_stats_get")
        return {f: getattr(st, f) for f, _ in _lib.fw_server_stats._fields_}

    def now(self):
        return lib().fw_server_now(self.h)

    def close(self):
        if self.h:
            lib().fw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
