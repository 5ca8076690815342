"""ctypes binding of libwcsim (include/wcsim.h).

Argument marshalling only: torch tensors supply device memory and the current CUDA stream;
every stage of the simulation runs in the library's CUDA kernels.  There is no CPU or
eager fallback: if libwcsim.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

from .synth import Depos, DriftParams, Geometry

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libwcsim.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "wcsim.h")

OK, EINVAL, ESHAPE, ENOMEM, ECUDA, ETIMEOUT, EDEVICE_CHECK = range(7)
STATUS_NAMES = {0: "WCSIM_OK", 1: "WCSIM_EINVAL", 2: "WCSIM_ESHAPE", 3: "WCSIM_ENOMEM",
                4: "WCSIM_ECUDA", 5: "WCSIM_ETIMEOUT", 6: "WCSIM_EDEVICE_CHECK"}
STAGES = ("prep", "rasterize", "rows_r2c", "wire_pass", "rows_c2r")
BWD_STAGES = ("bwd_zero", "bwd_rasterize", "bwd_r2c_S", "bwd_r2c_G", "bwd_wire_adjoint",
              "bwd_c2r_dS", "bwd_depo_adjoint")


class WcsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class CGeometry(ctypes.Structure):
    _fields_ = [("n_wires", ctypes.c_int32), ("n_imp", ctypes.c_int32),
                ("n_ticks", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("pitch_mm", ctypes.c_double), ("p0_mm", ctypes.c_double),
                ("tick_us", ctypes.c_double), ("t0_us", ctypes.c_double)]


class CParams(ctypes.Structure):
    _fields_ = [("v_mm_per_us", ctypes.c_double), ("DL_cm2_s", ctypes.c_double),
                ("DT_cm2_s", ctypes.c_double), ("lifetime_us", ctypes.c_double),
                ("nsigma", ctypes.c_double), ("fluctuate", ctypes.c_int32),
                ("plane_id", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("renormalize", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class CDepos(ctypes.Structure):
    _fields_ = [("p_mm", ctypes.c_void_p), ("t_us", ctypes.c_void_p),
                ("tdrift_us", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("id", ctypes.c_void_p), ("n", ctypes.c_int64)]


class CDepoGrads(ctypes.Structure):
    _fields_ = [("dq", ctypes.c_void_p), ("dp", ctypes.c_void_p), ("dt", ctypes.c_void_p),
                ("dsigma_L", ctypes.c_void_p), ("dsigma_T", ctypes.c_void_p),
                ("dglobal", ctypes.c_void_p)]


GRAD_NAMES = ("q", "p", "t", "sigma_L", "sigma_T")


class CTuneReport(ctypes.Structure):
    _fields_ = [("time_radix", ctypes.c_int32 * 8), ("rows_variant", ctypes.c_int32),
                ("wire_variant", ctypes.c_int32), ("depos_per_block", ctypes.c_int32),
                ("candidates_timed", ctypes.c_int32), ("ms_rasterize", ctypes.c_float),
                ("ms_rows", ctypes.c_float), ("ms_wire", ctypes.c_float),
                ("forward_fused", ctypes.c_int32), ("ms_forward_plain", ctypes.c_float),
                ("ms_forward_fused", ctypes.c_float), ("lanes_per_depo", ctypes.c_int32)]

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libwcsim.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
    L = ctypes.CDLL(_LIB_PATH)
    P, vp, i32, st = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
    sig = {
        "wcsim_plane_create": [P(CGeometry), vp, i32, i32, P(CParams), vp, P(vp)],
        "wcsim_plane_set_params": [vp, P(CParams)],
        "wcsim_plane_set_response": [vp, vp, vp],
        "wcsim_rasterize": [vp, P(CDepos), vp, vp],
        "wcsim_convolve": [vp, vp, vp, vp],
        "wcsim_run": [vp, P(CDepos), vp, vp],
        "wcsim_windows": [vp, P(CDepos), vp, vp],
        "wcsim_plane_check": [vp, vp, P(i32)],
        "wcsim_plane_set_timing": [vp, i32],
        "wcsim_plane_stage_times": [vp, P(ctypes.c_float), i32],
        "wcsim_plane_destroy": [vp],
        "wcsim_convolve_noalloc": [P(CGeometry), vp, i32, i32, vp, vp, vp],
        "wcsim_convolve_noalloc_check": [vp, P(i32)],
        "wcsim_convolve_adjoint": [vp, vp, vp, vp, vp, vp],
        "wcsim_rasterize_adjoint": [vp, P(CDepos), vp, P(CDepoGrads), vp],
        "wcsim_run_backward": [vp, P(CDepos), vp, P(CDepoGrads), vp, vp],
        "wcsim_batch_run": [i32, P(vp), P(CDepos), P(vp), vp],
        "wcsim_plane_autotune": [vp, P(CDepos), vp, P(CTuneReport)],
        "wcsim_plane_reserve_batch": [vp, i32],
        "wcsim_plane_set_wait_limit": [vp, ctypes.c_uint64],
        "wcsim_plane_set_noise": [vp, vp, i32, ctypes.c_uint64, vp],
        "wcsim_run_adc": [vp, P(CDepos), vp, vp],
        "wcsim_run_residual": [vp, P(CDepos), vp, vp, vp, vp],
        "wcsim_plane_set_digitizer": [vp, ctypes.c_float, ctypes.c_float, i32],
        "wcsim_plane_set_reuse_forward": [vp, i32],
        "wcsim_plane_set_forward": [vp, i32],
        "wcsim_plane_set_raster_tile": [vp, i32, i32],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.wcsim_last_error.restype = ctypes.c_char_p
    L.wcsim_last_error.argtypes = []
    L.wcsim_version.restype = ctypes.c_char_p
    L.wcsim_version.argtypes = []
    _lib = L
    return L


def header_functions(path: str = HEADER):
    """Names of the functions include/wcsim.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(wcsim_[a-z_0-9]+)\s*\(", txt)))


def check(status: int):
    if status != OK:
        raise WcsimError(status, lib().wcsim_last_error().decode())


def c_geometry(g: Geometry) -> CGeometry:
    return CGeometry(int(g.n_wires), int(g.n_imp), int(g.n_ticks), 0, float(g.pitch_mm),
                     float(g.p0_mm), float(g.tick_us), float(g.t0_us))


def c_params(p: DriftParams) -> CParams:
    return CParams(float(p.v_mm_per_us), float(p.DL_cm2_s), float(p.DT_cm2_s),
                   float(p.lifetime_us), float(p.nsigma), int(p.fluctuate),
                   int(p.plane_id) & 0xFFFFFFFF, int(p.seed) & 0xFFFFFFFFFFFFFFFF,
                   int(getattr(p, "renormalize", 0)), 0)


def _stream_handle(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


_DEPO_SERIAL = [0]


class DeviceDepos:
    """Depos resident on the GPU (torch tensors); keeps the tensors alive for the C struct.
    Each instance has a serial number, so that a plane can tell two depo sets apart even when
    the caching allocator gives the second the first one's addresses."""

    def __init__(self, p, t, td, q, ids):
        self.p, self.t, self.td, self.q, self.id = p, t, td, q, ids
        _DEPO_SERIAL[0] += 1
        self.serial = _DEPO_SERIAL[0]
        n = int(p.shape[0])
        for a in (p, t, td, q, ids):
            assert int(a.shape[0]) == n and a.is_cuda and a.is_contiguous()
        self.c = CDepos(p.data_ptr(), t.data_ptr(), td.data_ptr(), q.data_ptr(),
                        ids.data_ptr(), n)

    def __len__(self):
        return int(self.c.n)

    @classmethod
    def from_host(cls, d: Depos, device="cuda", non_blocking=False):
        import torch
        ids = torch.from_numpy(np.ascontiguousarray(d.id, np.uint32).view(np.int32))
        return cls(torch.from_numpy(np.ascontiguousarray(d.p, np.float64)).to(device, non_blocking=non_blocking),
                   torch.from_numpy(np.ascontiguousarray(d.t, np.float64)).to(device, non_blocking=non_blocking),
                   torch.from_numpy(np.ascontiguousarray(d.td, np.float64)).to(device, non_blocking=non_blocking),
                   torch.from_numpy(np.ascontiguousarray(d.q, np.float32)).to(device, non_blocking=non_blocking),
                   ids.to(device, non_blocking=non_blocking))


class Plane:
    """A wire plane: geometry, drift parameters and the detector response (Eq. 2)."""

    def __init__(self, geom: Geometry, params: DriftParams, response, n_fw: int = 0,
                 n_ft: int = 0, stream=None):
        import torch
        L = lib()
        self.geom, self.params = geom, params
        if not isinstance(response, torch.Tensor):
            response = torch.from_numpy(np.ascontiguousarray(response, np.complex64))
        if not response.is_cuda:
            response = response.cuda()
        response = response.contiguous()
        assert response.dtype == torch.complex64 and response.dim() == 3
        self.n_fw = n_fw or int(response.shape[1])
        self.n_ft = n_ft or int(response.shape[2])
        h = ctypes.c_void_p()
        check(L.wcsim_plane_create(ctypes.byref(c_geometry(geom)), response.data_ptr(),
                                   self.n_fw, self.n_ft, ctypes.byref(c_params(params)),
                                   _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().wcsim_plane_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: DriftParams):
        check(lib().wcsim_plane_set_params(self._h, ctypes.byref(c_params(params))))
        self.params = params

    def set_response(self, response, stream=None):
        check(lib().wcsim_plane_set_response(self._h, response.contiguous().data_ptr(),
                                             _stream_handle(stream)))
        self.response_serial = getattr(self, "response_serial", 0) + 1

    def _wave(self, out):
        import torch
        if out is None:
            out = torch.empty((self.geom.n_wires, self.geom.n_ticks), dtype=torch.float32,
                              device="cuda")
        assert out.dtype == torch.float32 and out.is_contiguous()
        return out

    def rasterize(self, depos: DeviceDepos, grid, stream=None):
        """Add every depo's patch into ``grid`` (float32 [n_wires*n_imp][n_ticks])."""
        assert grid.is_contiguous() and grid.numel() == self.geom.n_rows * self.geom.n_ticks
        check(lib().wcsim_rasterize(self._h, ctypes.byref(depos.c), grid.data_ptr(),
                                    _stream_handle(stream)))
        return grid

    def convolve(self, grid, out=None, stream=None):
        out = self._wave(out)
        check(lib().wcsim_convolve(self._h, grid.data_ptr(), out.data_ptr(),
                                   _stream_handle(stream)))
        return out

    def run(self, depos: DeviceDepos, out=None, stream=None):
        out = self._wave(out)
        check(lib().wcsim_run(self._h, ctypes.byref(depos.c), out.data_ptr(),
                              _stream_handle(stream)))
        self._last_run_serial = depos.serial
        return out

    def run_residual(self, depos: DeviceDepos, target, out=None, loss=None, stream=None):
        """M - target for the frame M of run() (float32 [n_wires, n_ticks] on the GPU) and,
        in `loss` (a float64 tensor of one element, made if None), L = 1/2 |M - target|^2;
        see wcsim_run_residual.  Returns (residual, loss)."""
        import torch
        out = self._wave(out)
        target = target.contiguous()
        if target.shape != out.shape or target.dtype != torch.float32 or not target.is_cuda:
            raise ValueError("target must be a float32 CUDA tensor of shape %s" % (tuple(out.shape),))
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
        check(lib().wcsim_run_residual(self._h, ctypes.byref(depos.c), target.data_ptr(),
                                       out.data_ptr(), loss.data_ptr(), _stream_handle(stream)))
        self._last_run_serial = depos.serial
        return out, loss

    def set_digitizer(self, gain: float, pedestal: float, bits: int):
        """ADC settings of run_adc; see wcsim_plane_set_digitizer."""
        check(lib().wcsim_plane_set_digitizer(self._h, float(gain), float(pedestal), int(bits)))

    def run_adc(self, depos: DeviceDepos, out=None, stream=None):
        """The frame of run() as ADC codes: a [n_wires, n_ticks] int16 tensor holding the
        uint16 codes' bits (view the host copy as uint16)."""
        import torch
        if out is None:
            out = torch.empty((self.geom.n_wires, self.geom.n_ticks), dtype=torch.int16,
                              device="cuda")
        assert out.dtype == torch.int16 and out.is_contiguous()
        assert tuple(out.shape) == (self.geom.n_wires, self.geom.n_ticks)
        check(lib().wcsim_run_adc(self._h, ctypes.byref(depos.c), out.data_ptr(),
                                  _stream_handle(stream)))
        return out

    # ------------------------------------------------------------ adjoint
    def _grads(self, n):
        import torch
        out = {k: torch.empty(n, dtype=torch.float32, device="cuda") for k in GRAD_NAMES}
        out["global"] = torch.empty(3, dtype=torch.float64, device="cuda")
        c = CDepoGrads(*[out[k].data_ptr() for k in GRAD_NAMES], out["global"].data_ptr())
        return out, c

    @staticmethod
    def _split_global(out):
        g = out.pop("global")
        out["DL"], out["DT"], out["lifetime"] = g[0], g[1], g[2]
        return out

    def _resp_buffer(self, want):
        import torch
        if not want:
            return None
        return torch.empty((self.geom.n_imp, self.n_fw, self.n_ft), dtype=torch.complex64,
                           device="cuda")

    def convolve_adjoint(self, grad_wave, grid, dgrid=None, want_resp=False, stream=None):
        """dL/dS (float32 grid shape) and, if asked, dL/dR (complex64) for dL/dM = grad_wave."""
        import torch
        if dgrid is None:
            dgrid = torch.empty_like(grid)
        dR = self._resp_buffer(want_resp)
        check(lib().wcsim_convolve_adjoint(self._h, grad_wave.contiguous().data_ptr(),
                                           grid.contiguous().data_ptr(), dgrid.data_ptr(),
                                           dR.data_ptr() if dR is not None else None,
                                           _stream_handle(stream)))
        return dgrid, dR

    def rasterize_adjoint(self, depos: DeviceDepos, dgrid, stream=None) -> dict:
        """Per-depo and global gradients given dL/dS (mean path, windows fixed)."""
        out, c = self._grads(len(depos))
        check(lib().wcsim_rasterize_adjoint(self._h, ctypes.byref(depos.c),
                                            dgrid.contiguous().data_ptr(), ctypes.byref(c),
                                            _stream_handle(stream)))
        return self._split_global(out)

    def backward(self, depos: DeviceDepos, grad_wave, want_resp=False, stream=None) -> dict:
        """Gradients of L with dL/dwave = grad_wave: per-depo q, p, t, sigma_L, sigma_T,
        global DL, DT, lifetime and (if asked) the response spectrum."""
        out, c = self._grads(len(depos))
        dR = self._resp_buffer(want_resp)
        if getattr(self, "_reuse", False) and getattr(self, "_last_run_serial", None) != depos.serial:
            # not the depo set of the last run (the library compares pointers only): drop the
            # kept spectra so that the backward recomputes them
            check(lib().wcsim_plane_set_reuse_forward(self._h, getattr(self, "_reuse_mode", 1)))
        check(lib().wcsim_run_backward(self._h, ctypes.byref(depos.c),
                                       grad_wave.contiguous().data_ptr(), ctypes.byref(c),
                                       dR.data_ptr() if dR is not None else None,
                                       _stream_handle(stream)))
        out = self._split_global(out)
        out["response"] = dR
        return out

    def autotune(self, depos: DeviceDepos, stream=None) -> dict:
        """Time kernel variants on `depos` and keep the fastest (see wcsim_plane_autotune)."""
        r = CTuneReport()
        check(lib().wcsim_plane_autotune(self._h, ctypes.byref(depos.c), _stream_handle(stream),
                                         ctypes.byref(r)))
        return {"time_radix": [x for x in r.time_radix if x], "rows_variant": r.rows_variant,
                "wire_variant": r.wire_variant, "depos_per_block": r.depos_per_block,
                "candidates_timed": r.candidates_timed, "ms_rasterize": r.ms_rasterize,
                "ms_rows": r.ms_rows, "ms_wire": r.ms_wire, "forward_fused": r.forward_fused,
                "ms_forward_plain": r.ms_forward_plain, "ms_forward_fused": r.ms_forward_fused,
                "lanes_per_depo": r.lanes_per_depo}

    def windows(self, depos: DeviceDepos, stream=None):
        import torch
        out = torch.empty((len(depos), 4), dtype=torch.int32, device="cuda")
        check(lib().wcsim_windows(self._h, ctypes.byref(depos.c), out.data_ptr(),
                                  _stream_handle(stream)))
        return out

    def check_flags(self, stream=None) -> int:
        f = ctypes.c_int32(0)
        st = lib().wcsim_plane_check(self._h, _stream_handle(stream), ctypes.byref(f))
        if st not in (OK, EDEVICE_CHECK):
            check(st)
        return int(f.value)

    def set_noise(self, amp=None, seed: int = 0, stream=None):
        """Eq. 1's noise for run / batch runs: amplitude spectrum amp (n_ft / 2 + 1 values,
        host) and Philox seed; None turns it off.  See wcsim_plane_set_noise."""
        import numpy as np
        if amp is None:
            check(lib().wcsim_plane_set_noise(self._h, None, 0, ctypes.c_uint64(0),
                                              _stream_handle(stream)))
            return
        a = np.ascontiguousarray(amp, np.float32)
        check(lib().wcsim_plane_set_noise(self._h, a.ctypes.data, a.size,
                                          ctypes.c_uint64(int(seed)), _stream_handle(stream)))

    def set_wait_limit(self, ns: int):
        """Limit (ns) of the device-side waits for bulk copies; see wcsim_plane_set_wait_limit."""
        check(lib().wcsim_plane_set_wait_limit(self._h, ctypes.c_uint64(int(ns))))

    def set_reuse_forward(self, enable: bool = True, keep_wire_spectra: bool = False):
        """Let backward() reuse the spectra of the preceding mean-path run() on the same depos
        and parameters (the depos must not change in between); see
        wcsim_plane_set_reuse_forward.  keep_wire_spectra: the forward also keeps the 2D
        spectra of S, from which a backward with want_resp=True takes dL/dR (mode 2).  The
        library recognises the depos by their device pointers and count only; this binding
        also requires the same DeviceDepos object (its serial), so tensors freed and
        reallocated at the same addresses are not mistaken for the forward's."""
        mode = (2 if keep_wire_spectra else 1) if enable else 0
        check(lib().wcsim_plane_set_reuse_forward(self._h, mode))
        self._reuse = bool(enable)
        self._reuse_mode = mode

    def set_forward(self, fused: bool = True):
        """Forward variant of run(): the rasterization fused into the time-axis transform
        (the grid never written), or the plain flow through the grid; see
        wcsim_plane_set_forward."""
        check(lib().wcsim_plane_set_forward(self._h, 1 if fused else 0))

    def set_raster_tile(self, depos_per_block: int, lanes_per_depo: int):
        """Rasterization tile (depos per CTA, lanes per depo); see
        wcsim_plane_set_raster_tile."""
        check(lib().wcsim_plane_set_raster_tile(self._h, int(depos_per_block),
                                                int(lanes_per_depo)))

    def set_timing(self, enable: bool = True):
        check(lib().wcsim_plane_set_timing(self._h, 1 if enable else 0))

    def stage_times(self, backward: bool = False) -> dict:
        names = STAGES + (BWD_STAGES if backward else ())
        arr = (ctypes.c_float * len(names))()
        check(lib().wcsim_plane_stage_times(self._h, arr, len(names)))
        return dict(zip(names, [float(x) for x in arr]))


def convolve_noalloc(geom: Geometry, response, grid, out=None, n_fw: int = 0, n_ft: int = 0,
                     stream=None):
    """Eq. 2 convolution through wcsim_convolve_noalloc: no device allocation inside the
    library (its scratch is a fixed static device array, shared by all calls on a device;
    calls must not overlap on the GPU).  `response`, `grid` and `out` are CUDA tensors."""
    import torch
    if out is None:
        out = torch.empty((geom.n_wires, geom.n_ticks), dtype=torch.float32, device="cuda")
    assert response.is_cuda and grid.is_cuda and out.is_cuda
    assert response.dtype == torch.complex64 and grid.dtype == torch.float32
    check(lib().wcsim_convolve_noalloc(ctypes.byref(c_geometry(geom)),
                                       response.contiguous().data_ptr(), int(n_fw), int(n_ft),
                                       grid.contiguous().data_ptr(), out.data_ptr(),
                                       _stream_handle(stream)))
    return out


def convolve_noalloc_check(stream=None) -> int:
    """Flag bits of the last convolve_noalloc call on the current device (waits for its
    stream; allocates nothing).  Raises WcsimError (ETIMEOUT) when a device-side wait of that
    call gave up, so part of its output is missing."""
    f = ctypes.c_int32(0)
    check(lib().wcsim_convolve_noalloc_check(_stream_handle(stream), ctypes.byref(f)))
    return int(f.value)


MAX_BATCH = 64


class Batch:
    """A fixed list of events (plane, device depos, output waveform) run with one
    wcsim_batch_run call.  Holds the marshalled C arrays so that the call can be repeated
    (or recorded in a CUDA graph) without rebuilding them."""

    def __init__(self, planes, depos, waves=None):
        import torch
        assert len(planes) == len(depos) <= MAX_BATCH
        self.planes, self.depos = list(planes), list(depos)
        if waves is None:
            waves = [torch.empty((p.geom.n_wires, p.geom.n_ticks), dtype=torch.float32,
                                 device="cuda") for p in self.planes]
        self.waves = list(waves)
        n = len(self.planes)
        self._p = (ctypes.c_void_p * n)(*[p.handle.value for p in self.planes])
        self._d = (CDepos * n)(*[d.c for d in self.depos])
        self._w = (ctypes.c_void_p * n)(*[w.data_ptr() for w in self.waves])
        counts = {}
        for p in self.planes:
            counts[id(p)] = counts.get(id(p), 0) + 1
        for p in {id(p): p for p in self.planes}.values():
            check(lib().wcsim_plane_reserve_batch(p.handle, counts[id(p)]))

    def run(self, stream=None):
        check(lib().wcsim_batch_run(len(self.planes), self._p, self._d, self._w,
                                    _stream_handle(stream)))
        return self.waves
