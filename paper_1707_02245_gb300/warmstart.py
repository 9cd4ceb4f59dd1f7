"""Learned warm start for the PDHG reconstruction: training pairs, training and
evaluation through the C ABI of include/pat_unet.h.

Loop control and argument marshalling only.  Every computation runs in the CUDA library:
- the reconstructions that produce the training pairs;
- the network's input features;
- the network's forward and backward passes and the Adam steps;
- the warm-started reconstructions.
PyTorch supplies device memory, streams and events.

The paper starts Algorithms 1 and 2 from zero.  Here a U-Net predicts the converged
iterates (u, v, r, s) from the data's backprojection.  q = K u - f follows from the
optimality condition of the data term (Sec. 3.2).  PDHG then runs from that state to the
same relative duality gap (Sec. 3.3.3) as a cold start.
"""
from __future__ import annotations

import time

import numpy as np

from . import (PAT_WARM_CHANNELS, Geometry, make_params, pat_forward, pat_reconstruct_batched,
               pat_unet_create, pat_unet_destroy, pat_unet_forward, pat_unet_get_params, pat_unet_num_params,
               pat_unet_set_params, pat_unet_train_step, pat_warm_start_features, pat_warm_start_state,
               pat_warm_start_target)

IN_CH = 8
OUT_CH = PAT_WARM_CHANNELS


class UNet:
    """Owner of a pat_unet handle."""

    def __init__(self, base_ch=32, levels=4, seed=0, in_ch=IN_CH, out_ch=OUT_CH):
        self.in_ch, self.out_ch, self.base_ch, self.levels = in_ch, out_ch, base_ch, levels
        self.handle = pat_unet_create(in_ch=in_ch, out_ch=out_ch, base_ch=base_ch, levels=levels, seed=seed)

    @property
    def num_params(self) -> int:
        return pat_unet_num_params(self.handle)

    def get_params(self) -> np.ndarray:
        return pat_unet_get_params(self.handle)

    def set_params(self, p) -> None:
        pat_unet_set_params(self.handle, p)

    def forward(self, x, batch, h, w, y, stream=None) -> None:
        pat_unet_forward(self.handle, x, batch, h, w, y, stream)

    def close(self):
        if getattr(self, "handle", None):
            pat_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _on(torch, stream):
    """Makes ``stream`` torch's current stream when it is a torch stream, so that the
    tensors allocated and filled here are ordered with the library's work on it."""
    import contextlib
    return torch.cuda.stream(stream) if isinstance(stream, torch.cuda.Stream) else contextlib.nullcontext()


def _ordered(fn):
    """Runs ``fn`` with its ``stream`` argument as torch's current stream."""
    import functools
    import inspect
    sig = inspect.signature(fn)

    @functools.wraps(fn)
    def wrap(*a, **kw):
        b = sig.bind(*a, **kw)
        with _on(b.arguments["torch"], b.arguments["stream"]):
            return fn(*a, **kw)
    return wrap


@_ordered
def simulate(torch, w: dict, device, stream):
    """Geometry and data f of a synthetic workload.  The data are K of the phantom on the
    2x finer grid with 2x the quadrature (no inverse crime, Sec. 5.2), plus Gaussian noise
    of std noise_level * max|clean|."""
    fine = Geometry(w["n_fine"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m_fine"])
    ph = torch.from_numpy(w["phantom_fine"].astype(np.float32)).to(device)
    clean = torch.empty(w["det_xy"].shape[0], w["n_t"], device=device)
    pat_forward(fine.handle, ph, clean, stream)
    noise = torch.from_numpy(w["noise"].astype(np.float32)).to(device)
    f = (clean + w["noise_level"] * clean.abs().max() * noise).contiguous()
    fine.close()
    return f


def state_sizes(w: dict) -> tuple[int, int]:
    """Lengths of the flat x = [u, v] and y = [q, r, s] of a TGV problem."""
    nn = w["n"] ** 2
    S = w["det_xy"].shape[0] * w["n_t"]
    return 3 * nn, S + 5 * nn


@_ordered
def make_pairs(torch, workloads: list[dict], geo: Geometry, device, stream, iters: int, tol: float = 0.0,
               batch: int = 16, gap_every: int = 10, step_ratio: float = 1.0):
    """Training pairs from PDHG itself.  Each problem is reconstructed (lockstep batches of
    ``batch``) for ``iters`` iterations, or until rel_gap <= tol.  Returns (features,
    targets, fs, infos):
    - features: count x N x N x 8, bf16;
    - targets: count x N x N x 8, FP32, the normalised (u, v, r, s);
    - fs: the data of each problem;
    - infos: the solver's reports.
    All workloads must share ``geo``'s geometry."""
    n = workloads[0]["n"]
    cnt = len(workloads)
    feats = torch.empty(cnt, n, n, IN_CH, dtype=torch.bfloat16, device=device)
    targs = torch.empty(cnt, n, n, OUT_CH, dtype=torch.float32, device=device)
    fs, infos = [], []
    nx, ny = state_sizes(workloads[0])
    for b0 in range(0, cnt, batch):
        ws = workloads[b0:b0 + batch]
        f_b = [simulate(torch, w, device, stream) for w in ws]
        xs = [torch.empty(nx, device=device) for _ in ws]
        ys = [torch.empty(ny, device=device) for _ in ws]
        us = [torch.empty(n, n, device=device) for _ in ws]
        prms = [make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], iters=iters, tol=tol,
                            gap_every=gap_every, step_ratio=step_ratio, x_out=x, y_out=y)
                for w, x, y in zip(ws, xs, ys)]
        infos += pat_reconstruct_batched([geo.handle] * len(ws), f_b, prms, us, stream)
        for k, (w, f, x, y, p) in enumerate(zip(ws, f_b, xs, ys, prms)):
            pat_warm_start_features(geo.handle, f, feats[b0 + k], IN_CH, stream)
            pat_warm_start_target(geo.handle, x, y, p, targs[b0 + k], OUT_CH, stream)
        fs += f_b
    return feats, targs, fs, infos


@_ordered
def train(torch, net: UNet, feats, targs, steps: int, batch: int, lr: float, ch_weight, stream, seed: int = 0,
          lr_final: float | None = None, log_every: int = 50):
    """Adam training on contiguous mini-batches of a shuffled order of whole batches.
    The learning rate decays by a cosine from lr to lr_final.  Returns the per-step
    losses that were read back (every ``log_every`` steps and the last) and the seconds
    spent."""
    cnt, n = feats.shape[0], feats.shape[1]
    nb = cnt // batch
    if nb == 0:
        raise ValueError("fewer samples than one batch")
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, device=device_of(feats))
    lr_final = lr * 0.05 if lr_final is None else lr_final
    log = []
    order = rng.permutation(nb)
    t0 = time.perf_counter()
    for s in range(steps):
        if s % nb == 0 and s:
            order = rng.permutation(nb)
        b = int(order[s % nb])
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * s / max(1, steps - 1)))
        pat_unet_train_step(net.handle, feats[b * batch:(b + 1) * batch], targs[b * batch:(b + 1) * batch],
                            ch_weight, batch, n, n, a, loss, stream)
        if s % log_every == 0 or s == steps - 1:
            log.append((s, float(loss.item())))
    torch.cuda.synchronize()
    return log, time.perf_counter() - t0


def device_of(t):
    return t.device




@_ordered
def predict_states(torch, net: UNet, geo: Geometry, feats, fs, params, device, stream, batch: int = 8):
    """Warm starts (x0, y0) for every problem: the network's forward pass on its
    features, in batches, then the state map.  Returns lists of x0 and y0 tensors."""
    cnt, n = feats.shape[0], feats.shape[1]
    pred = torch.empty(min(batch, cnt), n, n, OUT_CH, device=device)
    nx = 3 * n * n
    ny = fs[0].numel() + 5 * n * n
    x0s, y0s = [], []
    for b0 in range(0, cnt, batch):
        nb = min(batch, cnt - b0)
        net.forward(feats[b0:b0 + nb], nb, n, n, pred, stream)
        for k in range(nb):
            x0 = torch.empty(nx, device=device)
            y0 = torch.empty(ny, device=device)
            pat_warm_start_state(geo.handle, pred[k], OUT_CH, params[b0 + k], fs[b0 + k], x0, y0, stream)
            x0s.append(x0)
            y0s.append(y0)
    return x0s, y0s


@_ordered
def solve(torch, geo: Geometry, fs, workloads, device, stream, tol: float, max_iters: int, gap_every: int = 10,
          x0s=None, y0s=None, step_ratio: float = 1.0):
    """Solves every problem to rel_gap <= tol (cold, or from (x0s, y0s)) in one lockstep
    batch.  Returns (infos, images, seconds on the stream's events)."""
    n = workloads[0]["n"]
    us = [torch.empty(n, n, device=device) for _ in fs]
    prms = []
    for i, w in enumerate(workloads):
        kw = {}
        if x0s is not None:
            kw = dict(x0=x0s[i], y0=y0s[i])
        prms.append(make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], iters=max_iters, tol=tol,
                                gap_every=gap_every, step_ratio=step_ratio, **kw))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = pat_reconstruct_batched([geo.handle] * len(fs), fs, prms, us, stream)
    e1.record(stream)
    e1.synchronize()
    return infos, us, e0.elapsed_time(e1) / 1e3


def unet_flops(batch: int, h: int, w: int, base_ch: int = 32, levels: int = 4, in_ch: int = IN_CH,
               out_ch: int = OUT_CH) -> tuple[float, float]:
    """Multiply-add FLOPs (2 per MAC) of one forward pass and of one training step (forward,
    weight gradients, and input gradients of every conv but the first)."""
    ch = [base_ch * 2 ** l for l in range(levels)]
    convs = []   # (pixels per image, cin, cout)
    cin = in_ch
    for l in range(levels):
        px = (h >> l) * (w >> l)
        convs += [(px, cin, ch[l]), (px, ch[l], ch[l])]
        cin = ch[l]
    for l in range(levels - 2, -1, -1):
        px = (h >> l) * (w >> l)
        convs += [(px, ch[l + 1] + ch[l], ch[l]), (px, ch[l], ch[l])]
    convs.append((h * w, ch[0], out_ch))
    f = [2.0 * batch * px * 9 * ci * co for px, ci, co in convs]
    fwd = sum(f)
    return fwd, 3 * fwd - f[0]
