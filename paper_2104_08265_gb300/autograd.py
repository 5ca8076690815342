"""torch.autograd wrapper of the simulation: waveforms as a differentiable function of the
depo charges, positions, times and drift times, the diffusion constants, the electron
lifetime and the response spectrum.  Forward and backward both run in the CUDA library
(wcsim_run / wcsim_run_backward); this module only moves tensors across the C ABI and applies
the drift's chain rule for the drift time (Fig. 2: t_a = t + t_d, sigma = sqrt(2 D t_d),
Q' = Q exp(-t_d / lifetime)):
    dL/dt_d = dL/dt + dL/dsigma_L sigma_L / (2 t_d) + dL/dsigma_T sigma_T / (2 t_d)
              - dL/dQ Q / lifetime,
with the sigma terms 0 at t_d = 0 (where the library's sigma gradients are 0).  The
per-depo gradients with respect to sigma_L and sigma_T themselves are handed out through
the optional `sink` dict (keys sigma_L, sigma_T: float32 [n], per mm).

The backward pass differentiates the mean (fluctuation-free) waveform with every depo's bin
window held fixed, so a plane created with fluctuation on still gets the gradient of the
expected frame.  It runs with the parameters and the response of its own forward, even when
later forwards on the same plane changed them.  The depo tensors are saved for backward, so
autograd reports an in-place change made between the two; with
plane.set_reuse_forward(True) the backward of the plane's latest forward also reuses that
forward's spectra (fluctuation off).
"""
from __future__ import annotations

import dataclasses

import torch

from . import wcsim
from .synth import DriftParams


class WcsimFn(torch.autograd.Function):
    """wave = WcsimFn.apply(plane, q, p, t, td, ids, DL, DT, lifetime, response, sink).

    q: float32 [n]; p, t, td: float64 [n]; ids: int32 [n] (CUDA).  DL, DT [cm^2/s] and
    lifetime [us]: 0-d float64 tensors.  response: complex64 [n_imp][n_fw][n_ft] CUDA tensor
    or None (keep the plane's).  sink: None, or a dict that the backward fills with the
    per-depo sigma_L and sigma_T gradients.  Gradients flow to q, p, t, td, DL, DT, lifetime
    and response.
    """

    @staticmethod
    def forward(ctx, plane, q, p, t, td, ids, DL, DT, lifetime, response, sink=None):
        prm = dataclasses.replace(plane.params, DL_cm2_s=float(DL), DT_cm2_s=float(DT),
                                  lifetime_us=float(lifetime))
        plane.set_params(prm)
        if response is not None:
            plane.set_response(response)
        depos = wcsim.DeviceDepos(p.contiguous(), t.contiguous(), td.contiguous(),
                                  q.contiguous(), ids.contiguous())
        wave = plane.run(depos)
        ctx.plane = plane
        ctx.depos = depos
        ctx.prm = prm
        ctx.response_serial = getattr(plane, "response_serial", 0)
        ctx.save_for_backward(q, p, t, td, ids, response)
        ctx.want_resp = response is not None and response.requires_grad
        ctx.scalar_meta = [(x.dtype, x.device) for x in (DL, DT, lifetime)]
        ctx.sink = sink
        return wave

    @staticmethod
    def backward(ctx, grad_wave):
        plane = ctx.plane
        q, p, t, td, ids, response = ctx.saved_tensors   # (also checks the depos were not changed)
        if plane.params != ctx.prm:
            plane.set_params(ctx.prm)
        if getattr(plane, "response_serial", 0) != ctx.response_serial:
            if response is None:
                raise RuntimeError("the plane's response changed after this forward, which "
                                   "used the response the plane had then; pass it to simulate")
            plane.set_response(response)
        g = plane.backward(ctx.depos, grad_wave.contiguous().float(), want_resp=ctx.want_resp)
        (dl_t, dl_d), (dt_t, dt_d), (tau_t, tau_d) = ctx.scalar_meta
        if ctx.sink is not None:
            ctx.sink["sigma_L"] = g["sigma_L"]
            ctx.sink["sigma_T"] = g["sigma_T"]
        prm = ctx.prm
        tdd = td.double()
        live = tdd > 0
        safe = torch.where(live, tdd, torch.ones_like(tdd))
        # dsigma/dt_d = sigma / (2 t_d) = D / sigma, D in mm^2/us
        f_l = torch.where(live, torch.sqrt(2e-4 * prm.DL_cm2_s * safe) / (2 * safe), 0 * tdd)
        f_t = torch.where(live, torch.sqrt(2e-4 * prm.DT_cm2_s * safe) / (2 * safe), 0 * tdd)
        g_td = (g["t"].double() + g["sigma_L"].double() * f_l + g["sigma_T"].double() * f_t
                - g["q"].double() * q.double() / prm.lifetime_us)
        return (None, g["q"], g["p"].double(), g["t"].double(), g_td, None,
                g["DL"].to(dl_t).to(dl_d), g["DT"].to(dt_t).to(dt_d),
                g["lifetime"].to(tau_t).to(tau_d), g["response"], None)


def simulate(plane, depos: "wcsim.DeviceDepos", DL, DT, lifetime, response=None, sink=None):
    """Differentiable waveforms of `depos` on `plane` (see WcsimFn; `sink` receives the
    per-depo sigma_L / sigma_T gradients in the backward)."""
    return WcsimFn.apply(plane, depos.q, depos.p, depos.t, depos.td, depos.id, DL, DT,
                         lifetime, response, sink)
