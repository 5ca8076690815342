"""Fit of the global detector parameters over events sharded across ranks.

The loss is a sum over events, L = sum_e 1/2 |M_e - T_e|^2 (M_e the waveforms of event e,
T_e its target frame), so each global gradient (dL/dD_L, dL/dD_T, dL/dlifetime and dL/dR,
the response spectrum of Eq. 2) is a sum of per-event gradients.  Events are independent:
event e goes to rank e mod W, each rank runs the forward and backward of its own events
(the library's wcsim_run / wcsim_run_backward), and one all-reduce (sum) of the packed
global gradients gives every rank the gradient of the whole loss.  Every rank then applies
the same update, so the parameters stay identical across ranks without a broadcast.  Event
e keeps the fluctuation seed seed + e wherever it runs (the seeding of a batched run), so a
sharded fit sees the same events as a single-process one.

The reduction is torch.distributed's all_reduce (NCCL on GPUs, gloo on CPU); it is the only
exchange.  For NCCL, NVLink SHARP is switched off (NCCL_NVLS_ENABLE=0, unless the caller set
it) when the fit is built, before its first collective creates the communicator.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Callable, List, Optional, Sequence

import torch

from .synth import DriftParams

GLOBALS = ("DL", "DT", "lifetime")


def shard(n_events: int, world: int, rank: int) -> List[int]:
    """The global indices of the events rank `rank` of `world` runs: e = rank mod world."""
    if not (0 <= rank < world):
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return list(range(rank, n_events, world))


def event_params(params: DriftParams, e: int) -> DriftParams:
    """Event e's parameters: its fluctuation seed is the base seed + e."""
    return dataclasses.replace(params, seed=params.seed + e)


@dataclasses.dataclass
class FitState:
    """The fitted globals (identical on every rank): diffusion constants [cm^2/s], lifetime
    [us] and the response spectrum (complex64 [n_imp][n_fw][n_ft]) or None when not fitted."""
    DL: float
    DT: float
    lifetime: float
    response: Optional[torch.Tensor] = None


def gpu_event_gradient(plane, depos, target) -> Callable:
    """The per-event backward on the GPU: run event e on `plane` (wcsim_run_residual with the
    state's parameters and response: M - T and the loss), then wcsim_run_backward with
    dL/dM = M - T.  The backward takes
    the forward's spectra (wcsim_plane_set_reuse_forward; the run is on the mean path when
    params_e has fluctuate = 0), and, when the response is fitted, dL/dR from the 2D spectra
    the forward kept.  Returns a callable (state, params_e) -> (loss, {DL, DT, lifetime,
    response})."""

    def fn(state: FitState, params_e: DriftParams):
        plane.set_params(dataclasses.replace(params_e, DL_cm2_s=state.DL, DT_cm2_s=state.DT,
                                             lifetime_us=state.lifetime))
        if state.response is not None:
            plane.set_response(state.response)
        plane.set_reuse_forward(True, keep_wire_spectra=state.response is not None)
        G, loss_t = plane.run_residual(depos, target)      # M - T and 1/2 |M - T|^2
        g = plane.backward(depos, G, want_resp=state.response is not None)
        loss = float(loss_t)
        return loss, {"DL": float(g["DL"]), "DT": float(g["DT"]),
                      "lifetime": float(g["lifetime"]), "response": g["response"]}

    return fn


class ShardedFit:
    """Gradient descent on the globals over events sharded by rank.

    event_grads[i] is the per-event backward of the rank's i-th local event (shard order):
    (state, params_e) -> (loss_e, grads_e) with grads_e holding DL, DT, lifetime (floats) and
    response (a tensor, or None).  lr maps DL, DT, lifetime and response to step sizes.
    group: the torch.distributed process group (None: the default group, or a single
    process when torch.distributed is not initialised)."""

    def __init__(self, n_events: int, params: DriftParams, state: FitState,
                 event_grads: Sequence[Callable], lr: dict, group=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.events = shard(n_events, self.world, self.rank)
        if len(event_grads) != len(self.events):
            raise ValueError("rank %d runs %d events, got %d backward functions"
                             % (self.rank, len(self.events), len(event_grads)))
        self.params = params
        self.state = state
        self.event_grads = list(event_grads)
        self.lr = dict(lr)
        if self.dist and self.dist.get_backend(group) == "nccl":
            os.environ.setdefault("NCCL_NVLS_ENABLE", "0")

    def gradient(self):
        """(loss, gradients) of the whole loss over every rank's events: the local sums,
        packed and all-reduced once."""
        loss, g = 0.0, {k: 0.0 for k in GLOBALS}
        gr = None
        for e, fn in zip(self.events, self.event_grads):
            le, ge = fn(self.state, event_params(self.params, e))
            loss += le
            for k in GLOBALS:
                g[k] += ge[k]
            if ge.get("response") is not None:
                gr = ge["response"].clone() if gr is None else gr + ge["response"]
        dev = gr.device if gr is not None else torch.device("cpu")
        packed = torch.tensor([loss] + [g[k] for k in GLOBALS], dtype=torch.float64, device=dev)
        if self.dist and self.world > 1:
            if self.dist.get_backend(self.group) == "nccl" and packed.device.type == "cpu":
                packed = packed.cuda()
            self.dist.all_reduce(packed, group=self.group)
            if self.state.response is not None:
                if gr is None:
                    gr = torch.zeros_like(self.state.response)
                real = torch.view_as_real(gr)
                self.dist.all_reduce(real, group=self.group)
                gr = torch.view_as_complex(real)
        vals = packed.cpu().tolist()
        return vals[0], dict(zip(GLOBALS, vals[1:]), response=gr)

    def step(self):
        """One gradient step on every rank (the same update everywhere); returns the loss
        before the step."""
        loss, g = self.gradient()
        s = self.state
        s.DL -= self.lr.get("DL", 0.0) * g["DL"]
        s.DT -= self.lr.get("DT", 0.0) * g["DT"]
        s.lifetime -= self.lr.get("lifetime", 0.0) * g["lifetime"]
        if s.response is not None and g["response"] is not None:
            s.response = s.response - self.lr.get("response", 0.0) * g["response"].to(s.response.dtype)
        return loss
