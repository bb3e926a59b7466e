"""Seeded request media for the serving workload, generated on the device.

Each request of ``serving_stream`` (media.py) gets a Voronoi medium as in the
3D tissue workload: 64 seed points (32 in 2D), 8 classes whose (alpha0, y)
pairs are drawn from a table of pre-calibrated pairs (the paper's lookup
table of Sec. 3.2, here a small grid) and whose c, rho are uniform in
[1450, 1600] m/s and [900, 1100] kg/m^3, plus 2 % Gaussian jitter on c and
rho clipped at 3 sigma; a square planar source of half the lateral extent on
depth plane 24 with a 3 MHz Gaussian pulse; receivers on a stride-8 grid
two planes below the source.

Generation uses torch on the device (plane by plane nearest-seed search)
so that hundreds of requests up to 384^3 are ready in seconds.  Nothing here
performs any part of the simulation or of the calibration.
"""
from __future__ import annotations

import numpy as np

from .media import gaussian_pulse, plane_amplitude_rate

F0 = 3e6
DX = 1540.0 / (F0 * 12)
C_BOUND = 1600.0 * 1.06          # largest c after jitter: the CFL bound
DT = 0.4 * DX / C_BOUND
PML = 20


def lut_pairs(n_alpha=6, n_y=6, alpha0_range=(0.0022, 1.0), y_range=(0.4, 2.0)):
    """Grid of (alpha0, y) pairs the requests draw their classes from."""
    a = np.linspace(*alpha0_range, n_alpha)
    y = np.linspace(*y_range, n_y)
    return [(float(x), float(z)) for x in a for z in y]


def request_media(req, n_lut, device="cuda", n_class=8):
    """Maps of one request as torch tensors on ``device``: c, rho (float32),
    class_idx (int16 bit pattern of uint16 indices into the request's class
    list) and the request's class list as indices into the pair table, plus
    host source/receiver masks and the waveform."""
    import torch
    shape = tuple(req["shape"])
    nd = len(shape)
    rng = np.random.default_rng(req["seed"])
    n_seed = 64 if nd == 3 else 32
    seeds = rng.uniform(0.0, 1.0, size=(n_seed, nd)) * np.asarray(shape, dtype=np.float64)
    seed_class = rng.integers(0, n_class, size=n_seed)
    lut_idx = rng.integers(0, n_lut, size=n_class)
    cc = rng.uniform(1450.0, 1600.0, size=n_class)
    rr = rng.uniform(900.0, 1100.0, size=n_class)
    dev = torch.device(device)
    sd = torch.from_numpy(seeds).to(dev)
    scls = torch.from_numpy(seed_class).to(dev)
    cls = torch.empty(shape, dtype=torch.int16, device=dev)
    inner = [torch.arange(n, dtype=torch.float64, device=dev) + 0.5 for n in shape[1:]]
    grid = torch.meshgrid(*inner, indexing="ij")
    for k in range(shape[0]):
        d2 = (k + 0.5 - sd[:, 0]) ** 2
        for a, g in enumerate(grid):
            d2 = d2 + (g[..., None] - sd[:, a + 1]) ** 2
        cls[k] = scls[torch.argmin(d2, dim=-1)].to(torch.int16)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(req["seed"]))
    jc = torch.randn(shape, generator=gen, device=dev).clamp_(-3.0, 3.0)
    jr = torch.randn(shape, generator=gen, device=dev).clamp_(-3.0, 3.0)
    cl = cls.long()
    c = (torch.from_numpy(cc).float().to(dev)[cl] * (1.0 + 0.02 * jc)).contiguous()
    rho = (torch.from_numpy(rr).float().to(dev)[cl] * (1.0 + 0.02 * jr)).contiguous()
    src = np.zeros(shape, np.uint8)
    lat = [slice(n // 4, n // 4 + n // 2) for n in shape[1:]]
    src[tuple([24] + lat)] = 1
    rcv = np.zeros(shape, np.uint8)
    rcv[tuple([26] + [slice(n // 4, n // 4 + n // 2, 8) for n in shape[1:]])] = 1
    w = gaussian_pulse(F0, DT, req["n_steps"], plane_amplitude_rate(1e3, DX, nd, 1000.0, 1540.0))
    return dict(shape=shape, c=c, rho=rho, class_idx=cls, lut_idx=lut_idx, src_mask=src, rcv_mask=rcv,
                waves=w[None].astype(np.float32), n_steps=int(req["n_steps"]))
