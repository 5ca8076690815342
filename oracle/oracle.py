"""FP64 CPU oracle of the LArTPC signal-simulation hot path.

TEST INFRASTRUCTURE ONLY: the slow, plainly-correct reference the CUDA library is checked
against.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it.  It shares no code with the CUDA path; both only take arrays produced by the
seeded input generators.

Stages (paper Sec. 2.1.1, Eq. 1 and Eq. 2):

* ``rasterize``  -- drift, rasterization, optional fluctuation and scatter-add into the
  impact x tick grid S, in FP64 (``wcsim_oracle.c``).
* ``convolve``   -- Eq. 2 taken literally per impact position j: S_j = rows j, j+n_imp, ...
  of S, zero-padded to the spectrum size; M = Re IFFT2( sum_j R_j . FFT2(S_j) ), cropped to
  the frame.  The FFT is numpy's float64 FFT (a library primitive), and the response is the
  full supplied spectrum R_j (not a Hermitian half).
* ``convolve_adjoint`` -- gradients of L through that map for a given G = dL/dM:
  dS_j = Re IFFT2(conj(R_j) . FFT2(G)) and dR_j = conj(FFT2(S_j)) . FFT2(G) / (n_fw n_ft)
  (the gradient convention of complex tensors in PyTorch: dL/dRe + i dL/dIm).
* ``depo_grads`` -- per-depo chain rule through rasterization and drift (C code).
* ``noise``      -- Eq. 1's additive term N(t, x): per wire, the normalised inverse DFT of an
  amplitude spectrum times unit complex Gaussians drawn from Philox4x32-10 (C code for the
  draws, numpy's irfft for the transform).
* ``digitize``   -- M as ADC codes: clamp(floor(g M + p + 1/2), 0, 2^bits - 1) in FP32.

Pins (tests, not this file): erf telescoping and quadrature for the weights, brute-force
bin enumeration for the windows, direct circular-sum convolution on tiny grids, a point
depo reproducing the shifted response, linearity / superposition, Philox against an
independent library implementation, fluctuation mean / variance, and finite differences
for the adjoint.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wcsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = [os.environ.get("CC", "gcc"), "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [("n_wires", ctypes.c_int32), ("n_imp", ctypes.c_int32),
                ("n_ticks", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("pitch_mm", ctypes.c_double), ("p0_mm", ctypes.c_double),
                ("tick_us", ctypes.c_double), ("t0_us", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("v_mm_per_us", ctypes.c_double), ("DL_cm2_s", ctypes.c_double),
                ("DT_cm2_s", ctypes.c_double), ("lifetime_us", ctypes.c_double),
                ("nsigma", ctypes.c_double), ("fluctuate", ctypes.c_int32),
                ("plane_id", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("renormalize", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, f, u32, i64 = ctypes.c_double, ctypes.c_float, ctypes.c_uint32, ctypes.c_int64
            lib.og_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            lib.og_normal.argtypes = [u32, u32, ctypes.c_int]
            lib.og_normal.restype = d
            lib.og_bin_normal.argtypes = [i64, i64, u32, u32, P(u32)]
            lib.og_bin_normal.restype = d
            lib.og_bin_uniform.argtypes = [i64, i64, u32, u32, P(u32)]
            lib.og_bin_uniform.restype = d
            lib.og_binomial_draw.argtypes = [i64, d, d]
            lib.og_binomial_draw.restype = i64
            lib.og_noise_spectrum.argtypes = [ctypes.c_int32, ctypes.c_int32, u32, P(u32),
                                              P(d), P(d)]
            lib.og_noise_spectrum.restype = None
            lib.og_windows.argtypes = [P(_Geom), P(_Params), i64, P(d), P(d), P(d), P(f),
                                       P(i64)]
            lib.og_depo_weights.argtypes = [P(_Geom), P(_Params), d, d, d, f, P(d), P(d),
                                            P(d)]
            lib.og_depo_weights.restype = ctypes.c_int
            lib.og_rasterize.argtypes = [P(_Geom), P(_Params), i64, P(d), P(d), P(d), P(f),
                                         P(u32), P(d)]
            lib.og_rasterize.restype = ctypes.c_int
            lib.og_depo_grads.argtypes = [P(_Geom), P(_Params), i64, P(d), P(d), P(d), P(f),
                                          P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
            lib.og_depo_grads.restype = ctypes.c_int
            lib.og_rasterize_rows.argtypes = [P(_Geom), P(_Params), i64, P(d), P(d), P(d), P(f),
                                              P(u32), i64, P(i64), P(i64), P(d)]
            lib.og_rasterize_rows.restype = ctypes.c_int
            lib.og_bin_terms.argtypes = [P(_Geom), P(_Params), i64, P(d), P(d), P(d), P(f),
                                         P(u32), i64, i64, i64, P(i64), P(d), P(d), P(d), P(d)]
            lib.og_bin_terms.restype = i64
            lib.og_rasterize_mt.argtypes = [P(_Geom), P(_Params), i64, P(d), P(d), P(d), P(f),
                                            P(u32), ctypes.c_int, ctypes.c_void_p, P(d)]
            lib.og_rasterize_mt.restype = ctypes.c_int
            lib.og_patch_bytes.argtypes = []
            lib.og_patch_bytes.restype = i64
            _lib = lib
    return _lib


def _geom(g) -> _Geom:
    return _Geom(int(g.n_wires), int(g.n_imp), int(g.n_ticks), 0, float(g.pitch_mm),
                 float(g.p0_mm), float(g.tick_us), float(g.t0_us))


def _params(p) -> _Params:
    return _Params(float(p.v_mm_per_us), float(p.DL_cm2_s), float(p.DT_cm2_s),
                   float(p.lifetime_us), float(p.nsigma), int(p.fluctuate),
                   int(p.plane_id) & 0xFFFFFFFF, int(p.seed) & 0xFFFFFFFFFFFFFFFF,
                   int(getattr(p, "renormalize", 0)), 0)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _depo_arrays(d):
    p = np.ascontiguousarray(d.p, np.float64)
    t = np.ascontiguousarray(d.t, np.float64)
    td = np.ascontiguousarray(d.td, np.float64)
    q = np.ascontiguousarray(d.q, np.float32)
    ids = np.ascontiguousarray(d.id, np.uint32)
    return p, t, td, q, ids


# --------------------------------------------------------------------------- Philox
def philox4x32_10(ctr, key):
    """Philox4x32-10 block for one counter (4 x u32) and key (2 x u32)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.og_philox4x32_10(c, k, o)
    return [int(o[i]) for i in range(4)]


def normal_from_words(x0: int, x1: int, which: int = 0) -> float:
    """Box-Muller standard normal from two Philox words (FP64); which: 0 cos, 1 sin."""
    return float(_load().og_normal(int(x0) & 0xFFFFFFFF, int(x1) & 0xFFFFFFFF, int(which)))


def bin_normal(r: int, k: int, depo_id: int, plane_id: int, seed: int) -> float:
    """The standard normal that fluctuates bin (row r, tick k) of a depo."""
    key = (ctypes.c_uint32 * 2)(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return float(_load().og_bin_normal(int(r), int(k), int(depo_id) & 0xFFFFFFFF,
                                       int(plane_id) & 0xFFFFFFFF, key))


def bin_uniform(r: int, k: int, depo_id: int, plane_id: int, seed: int) -> float:
    """The uniform (23 bits) that draws the exact binomial of bin (row r, tick k) of a depo."""
    key = (ctypes.c_uint32 * 2)(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return float(_load().og_bin_uniform(int(r), int(k), int(depo_id) & 0xFFFFFFFF,
                                        int(plane_id) & 0xFFFFFFFF, key))


def binomial_draw(n: int, p: float, u: float) -> int:
    """Binomial(n, p) by inversion of its CDF at u (the smallest k with u < F(k))."""
    return int(_load().og_binomial_draw(int(n), float(p), float(u)))


# --------------------------------------------------------------------------- a1-a3
def windows(geom, params, depos) -> np.ndarray:
    """[n][4] int64: r_lo, r_hi, k_lo, k_hi of the bins each depo covers (-1 if none)."""
    lib = _load()
    p, t, td, q, _ = _depo_arrays(depos)
    out = np.empty((p.shape[0], 4), np.int64)
    lib.og_windows(ctypes.byref(_geom(geom)), ctypes.byref(_params(params)), p.shape[0],
                   _ptr(p, ctypes.c_double), _ptr(t, ctypes.c_double),
                   _ptr(td, ctypes.c_double), _ptr(q, ctypes.c_float),
                   _ptr(out, ctypes.c_int64))
    return out


def depo_weights(geom, params, p, t, td, q):
    """(Q', w_pitch, w_time) of one depo, or None if it covers no bin."""
    lib = _load()
    g = _geom(geom)
    n = g.n_wires * g.n_imp + g.n_ticks + 2
    wp = np.zeros(n); wt = np.zeros(n); qa = ctypes.c_double()
    ok = lib.og_depo_weights(ctypes.byref(g), ctypes.byref(_params(params)), float(p),
                             float(t), float(td), float(q), ctypes.byref(qa),
                             _ptr(wp, ctypes.c_double), _ptr(wt, ctypes.c_double))
    if not ok:
        return None
    w = windows(geom, params, _One(p, t, td, q))[0]
    return qa.value, wp[: w[1] - w[0] + 1].copy(), wt[: w[3] - w[2] + 1].copy()


class _One:
    def __init__(self, p, t, td, q):
        self.p = np.array([p], np.float64); self.t = np.array([t], np.float64)
        self.td = np.array([td], np.float64); self.q = np.array([q], np.float32)
        self.id = np.zeros(1, np.uint32)


def rasterize(geom, params, depos, threads: int = 1) -> np.ndarray:
    """Grid S [n_wires*n_imp][n_ticks] (float64) with every depo's patch added, in depo order.
    threads != 1 fills bands of rows on that many host threads (0: all), bit for bit the
    same grid."""
    lib = _load()
    p, t, td, q, ids = _depo_arrays(depos)
    grid = np.zeros((geom.n_wires * geom.n_imp, geom.n_ticks), np.float64)
    args = (ctypes.byref(_geom(geom)), ctypes.byref(_params(params)), p.shape[0],
            _ptr(p, ctypes.c_double), _ptr(t, ctypes.c_double), _ptr(td, ctypes.c_double),
            _ptr(q, ctypes.c_float), _ptr(ids, ctypes.c_uint32))
    if threads == 1:
        rc = lib.og_rasterize(*args, _ptr(grid, ctypes.c_double))
    else:
        scratch = np.empty(max(1, p.shape[0]) * int(lib.og_patch_bytes()), np.uint8)
        rc = lib.og_rasterize_mt(*args, int(threads), scratch.ctypes.data,
                                 _ptr(grid, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle: patch larger than its fixed buffer")
    return grid


def rasterize_rows(geom, params, depos, rows) -> np.ndarray:
    """Rows `rows` (distinct) of the grid rasterize() makes, bit for bit: [len(rows)][n_ticks]."""
    lib = _load()
    p, t, td, q, ids = _depo_arrays(depos)
    rows = np.ascontiguousarray(rows, np.int64)
    out = np.zeros((rows.shape[0], geom.n_ticks), np.float64)
    slot = np.empty(geom.n_wires * geom.n_imp, np.int64)
    rc = lib.og_rasterize_rows(ctypes.byref(_geom(geom)), ctypes.byref(_params(params)),
                               p.shape[0], _ptr(p, ctypes.c_double), _ptr(t, ctypes.c_double),
                               _ptr(td, ctypes.c_double), _ptr(q, ctypes.c_float),
                               _ptr(ids, ctypes.c_uint32), rows.shape[0],
                               _ptr(rows, ctypes.c_int64), _ptr(slot, ctypes.c_int64),
                               _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle: bad rows or patch larger than its fixed buffer")
    return out


def bin_terms(geom, params, depos, r: int, k: int, max_terms: int = 4096) -> dict:
    """The terms of grid bin (r, k), one per depo whose window holds it, in depo order:
    depo index, value added, and the trial count, p_b and uniform of its exact binomial draw
    (n_e = -1 where no draw is made)."""
    lib = _load()
    p, t, td, q, ids = _depo_arrays(depos)
    idx = np.zeros(max_terms, np.int64)
    val, n_e, pb, u = (np.zeros(max_terms) for _ in range(4))
    m = lib.og_bin_terms(ctypes.byref(_geom(geom)), ctypes.byref(_params(params)), p.shape[0],
                         _ptr(p, ctypes.c_double), _ptr(t, ctypes.c_double),
                         _ptr(td, ctypes.c_double), _ptr(q, ctypes.c_float),
                         _ptr(ids, ctypes.c_uint32), int(r), int(k), max_terms,
                         _ptr(idx, ctypes.c_int64), _ptr(val, ctypes.c_double),
                         _ptr(n_e, ctypes.c_double), _ptr(pb, ctypes.c_double),
                         _ptr(u, ctypes.c_double))
    if m < 0:
        raise ValueError("oracle: more terms than max_terms")
    return {"idx": idx[:m], "val": val[:m], "n_e": n_e[:m], "p": pb[:m], "u": u[:m]}


# --------------------------------------------------------------------------- a4-a6
def _split(grid, n_imp, n_fw, n_ft):
    """S_j zero-padded to (n_fw, n_ft) for each impact position j."""
    n_rows, n_t = grid.shape
    n_w = n_rows // n_imp
    out = []
    for j in range(n_imp):
        s = np.zeros((n_fw, n_ft), np.float64)
        s[:n_w, :n_t] = grid[j::n_imp, :]
        out.append(s)
    return out


def convolve(geom, response, grid) -> np.ndarray:
    """Eq. 2: M = Re IFFT2(sum_j R_j FFT2(S_j)) cropped to [n_wires][n_ticks] (float64)."""
    R = np.asarray(response).astype(np.complex128)
    n_imp, n_fw, n_ft = R.shape
    assert n_imp == geom.n_imp
    Mh = np.zeros((n_fw, n_ft), np.complex128)
    for j, s in enumerate(_split(np.asarray(grid, np.float64), n_imp, n_fw, n_ft)):
        Mh += R[j] * np.fft.fft2(s)
    M = np.fft.ifft2(Mh).real
    return M[: geom.n_wires, : geom.n_ticks].copy()


def run(geom, params, response, depos, threads: int = 1) -> np.ndarray:
    """Depos to per-wire waveforms: rasterize (on `threads` host threads), then convolve."""
    return convolve(geom, response, rasterize(geom, params, depos, threads))


# --------------------------------------------------------------------------- noise
def noise_spectrum(n_w: int, n_ft: int, plane_id: int, seed: int) -> np.ndarray:
    """xi [n_w][n_ft/2 + 1] complex128: the unit-mean-square complex Gaussians of the noise
    (Philox4x32-10 + Box-Muller; real at k = 0 and at the Nyquist frequency)."""
    nh = n_ft // 2 + 1
    re = np.zeros((n_w, nh), np.float64)
    im = np.zeros((n_w, nh), np.float64)
    key = (ctypes.c_uint32 * 2)(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    _load().og_noise_spectrum(int(n_w), int(n_ft), int(plane_id) & 0xFFFFFFFF, key,
                              _ptr(re, ctypes.c_double), _ptr(im, ctypes.c_double))
    return re + 1j * im


def noise(geom, amp, n_ft: int, plane_id: int, seed: int) -> np.ndarray:
    """Eq. 1's N(t, x), [n_wires][n_ticks] float64: per wire the normalised inverse DFT over
    n_ft points of A(k) xi(k) (A: n_ft/2 + 1 amplitudes, Hermitian extension), cropped to the
    frame."""
    amp = np.asarray(amp, np.float64)
    assert amp.shape == (n_ft // 2 + 1,)
    xi = noise_spectrum(geom.n_wires, n_ft, plane_id, seed)
    return np.fft.irfft(amp[None, :] * xi, n=n_ft, axis=1)[:, : geom.n_ticks].copy()


# --------------------------------------------------------------------------- digitization
def digitize(wave, gain: float, pedestal: float, bits: int) -> np.ndarray:
    """M as ADC codes (Eq. 1 reads M as "an ADC value"; the paper gives no digitizer):
    code = clamp(floor(g M + p + 1/2), 0, 2^bits - 1), uint16.  The rounding is an integer
    decision, so it is taken in FP32, one rounded operation at a time: x = fl(fl(g M) + p),
    code = floor(fl(x + 1/2))."""
    m = np.asarray(wave, np.float32)
    g = np.float32(gain)
    p = np.float32(pedestal)
    x = (g * m).astype(np.float32) + p
    x = np.asarray(x, np.float32) + np.float32(0.5)
    code = np.floor(np.asarray(x, np.float32))
    top = float((1 << int(bits)) - 1)
    return np.clip(code, 0.0, top).astype(np.uint16)


def convolve_adjoint(geom, response, grid, G):
    """(dS [n_rows][n_ticks], dR [n_imp][n_fw][n_ft]) for L with dL/dM = G."""
    R = np.asarray(response).astype(np.complex128)
    n_imp, n_fw, n_ft = R.shape
    g = np.zeros((n_fw, n_ft), np.float64)
    g[: geom.n_wires, : geom.n_ticks] = G
    Gh = np.fft.fft2(g)
    dS = np.zeros((geom.n_wires * n_imp, geom.n_ticks), np.float64)
    dR = np.empty_like(R)
    for j, s in enumerate(_split(np.asarray(grid, np.float64), n_imp, n_fw, n_ft)):
        dS[j::n_imp, :] = np.fft.ifft2(np.conj(R[j]) * Gh).real[: geom.n_wires, : geom.n_ticks]
        dR[j] = np.conj(np.fft.fft2(s)) * Gh / (n_fw * n_ft)
    return dS, dR


# --------------------------------------------------------------------------- a7
def depo_grads(geom, params, depos, dS):
    """Per-depo dL/d(Q, p, t, sigma_L, sigma_T) and dL/d(D_L, D_T, tau) given dL/dS."""
    lib = _load()
    p, t, td, q, _ = _depo_arrays(depos)
    n = p.shape[0]
    dS = np.ascontiguousarray(dS, np.float64)
    outs = [np.zeros(n) for _ in range(5)]
    glob = np.zeros(3)
    rc = lib.og_depo_grads(ctypes.byref(_geom(geom)), ctypes.byref(_params(params)), n,
                           _ptr(p, ctypes.c_double), _ptr(t, ctypes.c_double),
                           _ptr(td, ctypes.c_double), _ptr(q, ctypes.c_float),
                           _ptr(dS, ctypes.c_double),
                           *[_ptr(o, ctypes.c_double) for o in outs],
                           _ptr(glob, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle: patch larger than its fixed buffer")
    names = ("q", "p", "t", "sigma_L", "sigma_T")
    res = dict(zip(names, outs))
    res.update(DL=glob[0], DT=glob[1], lifetime=glob[2])
    return res


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
