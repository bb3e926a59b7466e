"""torch.autograd.Function over the C ABI: receiver traces as a function of
the sound-speed map c(x) and the attenuation map alpha0(x).

Forward: fw_run on a medium built from the maps; backward: fw_gradient (the
hand-written adjoint kernels, checkpointed recomputation) with the incoming
dL/dtraces.  Argument marshalling only: every step runs in the library.

Two ways to build the medium:

* ``classes`` given (class map, list of fw_relax_params, alpha0 of each
  class): fw_create_medium_classes; alpha0 must equal the class value at
  every voxel (the gradient is taken there);
* otherwise fw_create_medium from the maps (every distinct (alpha0, y)
  pair calibrated on the host).

The gradient with respect to alpha0 follows the library's reading: the d of
a voxel's mechanisms scale with alpha0(x) / alpha0_class (kappa and alpha
fixed); see fw_gradient.

Lifetime: the forward keeps its medium (device memory) for the backward.
The backward runs once (``once_differentiable``): it releases the medium,
and a second backward through the same graph (retain_graph=True) raises.  A
forward whose inputs need no gradient releases its medium at once; one whose
backward never runs releases it when autograd frees the graph (the Medium's
finaliser).
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import Medium


class FullwaveSim(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, alpha0, setup):
        """setup: dict with shape, dx, dt, rho, n_steps, src_mask, waves,
        rcv_mask and optionally wave_of, pml, transition, f0, storage ('f32'
        or 'f64'), checkpoint, classes=(class_idx, params, alpha0_class) or
        y and n_mech (with fit options in fit_kw)."""
        f64 = setup.get("storage", "f32") == "f64"
        dev = c.device
        common = dict(dt=setup["dt"], pml=setup.get("pml", 0), transition=setup.get("transition", 0),
                      f0=setup.get("f0", 3e6), storage=setup.get("storage", "f32"))
        if setup.get("classes") is not None:
            cls, params, a0c = setup["classes"]
            want = torch.as_tensor(a0c, dtype=alpha0.dtype, device=alpha0.device)[
                torch.as_tensor(cls, dtype=torch.long, device=alpha0.device)]
            if not torch.equal(want, alpha0.detach()):
                raise ValueError("alpha0 must equal the class values when the medium is built from classes")
            m = Medium.from_classes(setup["shape"], setup["dx"], c.detach(), setup["rho"], cls, params, **common)
        else:
            m = Medium.from_maps(setup["shape"], setup["dx"], c.detach(), setup["rho"], alpha0.detach(),
                                 setup["y"], n_mech=setup.get("n_mech", 2), **common, **setup.get("fit_kw", {}))
        m.set_sources(setup["src_mask"], setup["waves"], setup.get("wave_of"))
        m.set_receivers(setup["rcv_mask"], setup["n_steps"])
        start = m.save_state()
        m.run(setup["n_steps"])
        traces = torch.as_tensor(m.receivers(f64=f64)).to(dev)
        if not (c.requires_grad or alpha0.requires_grad):
            m.close()                 # nothing can call backward: release the device memory now
            m = None
        ctx.medium, ctx.start, ctx.setup, ctx.f64 = m, start, setup, f64
        ctx.dtypes = (c.dtype, alpha0.dtype)
        ctx.save_for_backward(alpha0)
        return traces

    @staticmethod
    @once_differentiable
    def backward(ctx, grad_traces):
        (alpha0,) = ctx.saved_tensors
        m, setup = ctx.medium, ctx.setup
        if m is None:
            raise RuntimeError("FullwaveSim.backward runs once per forward: the first backward released the "
                               "medium; run the forward again for another gradient")
        dt = torch.float64 if ctx.f64 else torch.float32
        m.load_state(ctx.start)
        gc = torch.empty(setup["shape"], dtype=dt, device=grad_traces.device)
        ga = torch.empty(setup["shape"], dtype=dt, device=grad_traces.device)
        m.gradient(setup["n_steps"], grad_traces.detach().to(dt).contiguous(), alpha0=alpha0.detach().to(dt),
                   checkpoint=setup.get("checkpoint", 0), f64=ctx.f64, out=(gc, ga))
        m.close()
        ctx.medium = None
        return gc.to(ctx.dtypes[0]), ga.to(ctx.dtypes[1]), None


def simulate(c, alpha0, setup):
    """traces = FullwaveSim(c, alpha0) with autograd support."""
    return FullwaveSim.apply(c, alpha0, setup)
