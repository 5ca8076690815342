"""Seeded synthetic inputs for the LArTPC signal-simulation path.

This module only *generates inputs*: plane geometries, drift parameters, ionization
depositions ("depos") on straight tracks and the precomputed detector-response spectra
R(omega_t, omega_x) of Eq. 2.  It holds none of the simulation arithmetic (no drift, no
diffusion, no rasterization, no convolution); both the CUDA path and the FP64 oracle take
what it produces as plain arrays.

The paper's inputs (CORSIKA + Geant4 cosmic-ray depos produced with LArSoft, Sec. 4.3.2) are
not available, so tracks of the same shape stand in for them:

* depos lie on straight tracks, ordered along each track;
* charge per depo is lognormal with median 6000 electrons and sigma_ln = 0.3;
* drift time is uniform in [0, t_max] at the track end points and linear along the track;
* every stream is numpy PCG64 seeded with ``1000 + workload index``.

Units throughout: mm, microseconds, electrons; diffusion constants in cm^2/s.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict

import numpy as np

__all__ = [
    "Geometry", "DriftParams", "Depos", "Workload", "WORKLOADS",
    "track_depos", "event_depos_3d", "project_depos", "make_response", "make_workload",
]


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Plane geometry: rows are impact positions (n_imp per wire pitch), columns are ticks.

    Row r covers pitch coordinate [p0 + r*d, p0 + (r+1)*d) with d = pitch/n_imp; wire w owns
    rows w*n_imp .. w*n_imp + n_imp - 1.  Tick k covers [t0 + k*tick, t0 + (k+1)*tick).
    """
    n_wires: int
    n_imp: int
    n_ticks: int
    pitch_mm: float
    p0_mm: float = 0.0
    tick_us: float = 0.5
    t0_us: float = 0.0

    @property
    def n_rows(self) -> int:
        return self.n_wires * self.n_imp


@dataclasses.dataclass(frozen=True)
class DriftParams:
    """Drift / diffusion / lifetime / rasterization / fluctuation parameters."""
    v_mm_per_us: float = 1.6
    DL_cm2_s: float = 4.0
    DT_cm2_s: float = 8.8
    lifetime_us: float = 10000.0
    nsigma: float = 3.0
    fluctuate: int = 0       # 0 mean, 1 normal approximation, 2 exact binomial
    seed: int = 0
    plane_id: int = 0
    renormalize: int = 0     # 1: each axis divided by its n-sigma window's mass (unclipped)


@dataclasses.dataclass
class Depos:
    """Structure-of-arrays depos: p (f64 mm), t (f64 us), td (f64 us), q (f32 e-), id (u32)."""
    p: np.ndarray
    t: np.ndarray
    td: np.ndarray
    q: np.ndarray
    id: np.ndarray

    def __len__(self) -> int:
        return int(self.p.shape[0])

    def subset(self, idx) -> "Depos":
        return Depos(self.p[idx].copy(), self.t[idx].copy(), self.td[idx].copy(),
                     self.q[idx].copy(), self.id[idx].copy())


def _charges(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.lognormal(mean=math.log(6000.0), sigma=0.3, size=n).astype(np.float32)


def track_depos(rng: np.random.Generator, n_tracks: int, per_track: int, p_range: float,
                td_max: float) -> Depos:
    """Depos on ``n_tracks`` straight tracks in the (pitch, drift-time) plane.

    Both end points of each track are uniform in [0, p_range) x [0, td_max]; depo i of a
    track sits at fraction (i + 0.5)/per_track between them.
    """
    ps, tds = [], []
    for _ in range(n_tracks):
        a = rng.uniform(0.0, p_range, size=2)
        b = rng.uniform(0.0, td_max, size=2)
        f = (np.arange(per_track, dtype=np.float64) + 0.5) / per_track
        ps.append(a[0] + (a[1] - a[0]) * f)
        tds.append(b[0] + (b[1] - b[0]) * f)
    p = np.concatenate(ps)
    td = np.concatenate(tds)
    n = p.shape[0]
    return Depos(p=p, t=np.zeros(n), td=td, q=_charges(rng, n),
                 id=np.arange(n, dtype=np.uint32))


def event_depos_3d(rng: np.random.Generator, n_total: int, n_tracks: int, n_segments: int,
                   box_mm=(3600.0, 1200.0, 3000.0)):
    """3D depos (x = drift distance, y = along-wire height, z = beam) for a full event.

    ``n_segments`` isotropic short segments of length U[5, 50] mm carry round(len / 1 mm)
    depos each; ``n_tracks`` long tracks between two uniform points share the remainder.
    Returns (x, y, z, q) with x in mm of drift.
    """
    xs, ys, zs = [], [], []
    box = np.asarray(box_mm)
    used = 0
    for _ in range(n_segments):
        length = rng.uniform(5.0, 50.0)
        k = max(1, int(round(length)))
        c = rng.uniform(0.0, 1.0, size=3) * box
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        f = ((np.arange(k) + 0.5) / k - 0.5) * length
        pts = c[None, :] + f[:, None] * d[None, :]
        pts = np.clip(pts, 0.0, box)
        xs.append(pts[:, 0]); ys.append(pts[:, 1]); zs.append(pts[:, 2])
        used += k
    remain = max(0, n_total - used)
    counts = np.full(n_tracks, remain // n_tracks)
    counts[: remain % n_tracks] += 1
    for c in counts:
        a = rng.uniform(0.0, 1.0, size=3) * box
        b = rng.uniform(0.0, 1.0, size=3) * box
        f = (np.arange(c) + 0.5) / max(c, 1)
        pts = a[None, :] + f[:, None] * (b - a)[None, :]
        xs.append(pts[:, 0]); ys.append(pts[:, 1]); zs.append(pts[:, 2])
    x = np.concatenate(xs); y = np.concatenate(ys); z = np.concatenate(zs)
    return x, y, z, _charges(rng, x.shape[0])


def project_depos(x, y, z, q, angle_deg: float, v_mm_per_us: float, p_offset: float = 0.0
                  ) -> Depos:
    """Pitch coordinate of each 3D depo for wires at ``angle_deg`` from vertical."""
    a = math.radians(angle_deg)
    p = z * math.cos(a) + y * math.sin(a) + p_offset
    td = x / v_mm_per_us
    n = p.shape[0]
    return Depos(p=p.astype(np.float64), t=np.zeros(n), td=td.astype(np.float64),
                 q=np.asarray(q, np.float32), id=np.arange(n, dtype=np.uint32))


def _electronics(tick_us: float, n: int, tau_s: float = 0.5) -> np.ndarray:
    t = np.arange(n) * tick_us
    h = (t / tau_s) ** 4 * np.exp(-t / tau_s)
    return h / h.sum()


def make_response(geom: Geometry, kind: str = "collection", n_fw: int | None = None,
                  n_ft: int | None = None, span_wires: int = 10, span_ticks: int = 200,
                  sigma_f_us: float = 1.0, t_c_us: float = 10.0, backend: str = "numpy"):
    """Synthetic response spectra R_j(omega_x, omega_t), complex64 [n_imp][n_fw][n_ft].

    Field response per impact row j and wire offset dw in [-span, span]:
    collection = exp(-(t-t_c)^2 / 2 s^2) * exp(-|x|/pitch); induction is the bipolar
    -((t-t_c)/s) * exp(-(t-t_c)^2 / 2 s^2) * exp(-|x|/pitch), with x = dw*pitch - offset_j
    and offset_j = ((j + 0.5)/n_imp - 0.5) * pitch.  It is convolved in time with a
    4th-order semi-Gaussian shaper (t/tau)^4 exp(-t/tau), tau = 0.5 us (2 us peaking),
    normalised to unit sum, truncated to ``span_ticks`` ticks, placed at
    (dw mod n_fw, tick) and transformed with a float64 2D FFT, then rounded to complex64.
    backend="torch" does the float64 FFT with torch on the current CUDA device and returns
    a CUDA complex64 tensor (same values up to float64 rounding; for large benchmark planes).
    """
    n_fw = geom.n_wires if n_fw is None else n_fw
    n_ft = geom.n_ticks if n_ft is None else n_ft
    nt = min(span_ticks, n_ft)
    t = np.arange(nt) * geom.tick_us
    h = _electronics(geom.tick_us, nt)
    g = np.exp(-0.5 * ((t - t_c_us) / sigma_f_us) ** 2)
    if kind == "collection":
        ft = g
    elif kind == "induction":
        ft = -((t - t_c_us) / sigma_f_us) * g
    else:
        raise ValueError(kind)
    ft = np.convolve(ft, h)[:nt]
    if backend == "torch":
        import torch
        out = torch.empty((geom.n_imp, n_fw, n_ft), dtype=torch.complex64, device="cuda")
    else:
        out = np.empty((geom.n_imp, n_fw, n_ft), dtype=np.complex64)
    for j in range(geom.n_imp):
        off = ((j + 0.5) / geom.n_imp - 0.5) * geom.pitch_mm
        real = np.zeros((n_fw, n_ft), dtype=np.float64)
        for dw in range(-span_wires, span_wires + 1):
            x = dw * geom.pitch_mm - off
            real[dw % n_fw, :nt] += ft * math.exp(-abs(x) / geom.pitch_mm)
        if backend == "torch":
            out[j] = torch.fft.fft2(torch.from_numpy(real).cuda()).to(torch.complex64)
        else:
            out[j] = np.fft.fft2(real).astype(np.complex64)
    return out


@dataclasses.dataclass
class Workload:
    """One named workload: plane geometries, their drift parameters and depos."""
    name: str
    planes: list            # list of (Geometry, DriftParams, response kind, Depos)
    description: str


def batch_events(rng: np.random.Generator, n_events: int = 64, lo: float = 1e3, hi: float = 5e5,
                 wires=(480, 800, 960), ticks=(2000, 6000, 9600), scale: float = 1.0):
    """Independent events for a batched run: each draws a plane (wires x ticks uniform from
    the lists, 4.7 mm pitch, 10 impacts, collection or induction response) and a
    log-uniform depo count in [lo, hi] (times `scale`) on tracks of up to 2500 depos with
    drift time uniform in [0, 0.75 n_ticks tick]."""
    events = []
    for _ in range(n_events):
        g = Geometry(n_wires=int(rng.choice(wires)), n_imp=10, n_ticks=int(rng.choice(ticks)),
                     pitch_mm=4.7)
        kind = "collection" if rng.uniform() < 0.5 else "induction"
        n = max(1, int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))) * scale)))
        n_tracks = max(1, -(-n // 2500))
        d = track_depos(rng, n_tracks, -(-n // n_tracks), g.n_wires * g.pitch_mm,
                        0.75 * g.n_ticks * g.tick_us)
        d = d.subset(slice(0, n))
        events.append((g, kind, d))
    return events


# Workload table.  Index i is seeded with 1000 + i (depos) and 0x5EED0000 + i (fluctuation).
WORKLOADS: Dict[str, int] = {
    "plane128-2k": 0,          # 128 wires x 1024 ticks, 2,000 depos, fluctuation off
    "plane960-100k": 1,        # 960 wires x 6000 ticks, 100,000 depos, fluctuation on
    "event3p-1m": 2,           # 800 + 800 + 960 wires x 6000 ticks, 1,000,000 depos
    "fit960-100k": 3,          # 960 x 6000 plane, 100,000 depos, fluctuation off (fit target)
    "batch64": 4,              # 64 events, mixed planes, log-uniform 1e3..5e5 depos
}


def make_workload(name: str, n_depos: int | None = None) -> Workload:
    """Build a named workload; ``n_depos`` optionally overrides the depo count."""
    idx = WORKLOADS[name]
    rng = np.random.Generator(np.random.PCG64(1000 + idx))
    fseed = 0x5EED0000 + idx
    if name == "plane128-2k":
        g = Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
        n = 2000 if n_depos is None else n_depos
        per = max(1, n // 4)
        d = track_depos(rng, 4, per, g.n_wires * g.pitch_mm, 500.0)
        prm = DriftParams(fluctuate=0, seed=fseed)
        return Workload(name, [(g, prm, "collection", d)],
                        "1 plane 128 wires x 3 mm, 1024 ticks x 0.5 us, 4 tracks x 500 depos")
    if name in ("plane960-100k", "fit960-100k"):
        g = Geometry(n_wires=960, n_imp=10, n_ticks=6000, pitch_mm=4.7)
        n = 100000 if n_depos is None else n_depos
        per = max(1, n // 40)
        d = track_depos(rng, 40, per, g.n_wires * g.pitch_mm, 2250.0)
        fl = 1 if name == "plane960-100k" else 0
        prm = DriftParams(fluctuate=fl, seed=fseed)
        return Workload(name, [(g, prm, "collection", d)],
                        "1 plane 960 wires x 4.7 mm, 6000 ticks x 0.5 us, 40 tracks x 2500 depos")
    if name == "event3p-1m":
        n = 1000000 if n_depos is None else n_depos
        x, y, z, q = event_depos_3d(rng, n, 200, min(5000, max(1, n // 200)))
        planes = []
        for pid, (nw, ang, kind) in enumerate(((800, 35.7, "induction"),
                                               (800, -35.7, "induction"),
                                               (960, 0.0, "collection"))):
            g = Geometry(n_wires=nw, n_imp=10, n_ticks=6000, pitch_mm=4.7)
            off = 1200.0 * math.sin(math.radians(35.7)) if ang < 0 else 0.0
            d = project_depos(x, y, z, q, ang, 1.6, p_offset=off)
            prm = DriftParams(fluctuate=1, seed=fseed, plane_id=pid)
            planes.append((g, prm, kind, d))
        return Workload(name, planes, "3 planes (800 U, 800 V, 960 W) x 6000 ticks")
    if name == "batch64":
        evs = batch_events(rng, 64, scale=1.0 if n_depos is None else n_depos / 5.1e6)
        planes = [(g, DriftParams(fluctuate=1, seed=fseed), kind, d) for g, kind, d in evs]
        return Workload(name, planes, "64 events, planes 480/800/960 wires x 2000/6000/9600 ticks")
    raise KeyError(name)
