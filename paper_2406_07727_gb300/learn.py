"""Learned ordering of intermediate vertices (training driver).

The network is the library's ordering MLP (256 bfloat16 features [e_x[0:128];
e_endpoint[0:128]] -> 256 ReLU units -> 1).  It is trained to predict the
slack of the search's provable row bound for an intermediate vertex x: the
best fp32 path score through x minus that bound, both produced by plain
(exact, unpruned) runs of the search (``mhr_training_labels``).  At query
time the library sorts the rows it scans into 64 levels of their bound and,
inside a level, by the predicted slack (rows predicted closest to their bound
first), so the K-th score of a query rises early while whole work items can
still be skipped; pruning stays bound-based, so results never change.

This module only drives: data movement, shuffling and the epoch loop run on
the host; labels, features, forward, backward and Adam run in the library's
kernels.  torch provides device buffers.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import _mhr

N_W1 = 256 * 256
N_PARAMS = N_W1 + 256 + 256 + 1


class OrderingMLP:
    """Device-resident fp32 master parameters, their bf16 W1 copy and Adam state.
    Parameter layout: [W1 (256x256 row-major) | b1 (256) | w2 (256) | b2 (1)]."""

    def __init__(self, params=None, seed: int = 0):
        import torch
        if params is None:
            g = np.random.default_rng([seed, 7])
            p = np.zeros(N_PARAMS, dtype=np.float32)
            p[:N_W1] = g.standard_normal(N_W1).astype(np.float32) * np.float32(math.sqrt(2.0 / 256))
            p[N_W1 + 256:N_W1 + 512] = g.standard_normal(256).astype(np.float32) * np.float32(1 / 16)
            params = p
        self.params = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
        self.W1b = torch.empty(N_W1, dtype=torch.int16, device="cuda")
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.step = 0
        self.refresh()

    def refresh(self):
        _mhr.mhr_mlp_to_bf16(self.params[:N_W1], self.W1b)

    def struct(self) -> _mhr.MLP:
        base = self.params.data_ptr()
        m = _mhr.MLP()
        m.W1 = self.W1b.data_ptr()
        m.b1 = base + 4 * N_W1
        m.w2 = base + 4 * (N_W1 + 256)
        m.b2 = base + 4 * (N_W1 + 512)
        m._keep = self  # keep the tensors alive while the struct is in use
        return m

    def numpy(self) -> np.ndarray:
        return self.params.cpu().numpy()

    def fold_target_scale(self, mean: float, std: float):
        """y_raw = y_norm * std + mean, folded into w2 and b2."""
        p = self.numpy()
        p[N_W1 + 256:N_W1 + 512] *= np.float32(std)
        p[N_W1 + 512] = p[N_W1 + 512] * np.float32(std) + np.float32(mean)
        self.params.copy_(__import__("torch").from_numpy(p))
        self.refresh()


@dataclass
class TrainReport:
    rows: int
    epochs: int
    loss_first: float
    loss_last: float
    target_mean: float
    target_std: float


def collect_labels(G, S, T, queries_per_call: int = 256, cap: int = 1 << 22):
    """Training rows from plain runs: (near_v, end_v, slack target) on the host."""
    nv, ev, tg = [], [], []
    for i in range(0, len(S), queries_per_call):
        s, t = S[i:i + queries_per_call], T[i:i + queries_per_call]
        ok = s != t
        s, t = s[ok], t[ok]
        if len(s) == 0:
            continue
        try:
            a, b, own, best = _mhr.mhr_training_labels(G, s, t, cap)
        except _mhr.MhrError as e:
            if e.status != _mhr.MHR_ERANGE:
                raise
            a, b, own, best = _mhr.mhr_training_labels(G, s, t, cap * 8)
        nv.append(a.cpu().numpy().view(np.uint32))
        ev.append(b.cpu().numpy().view(np.uint32))
        tg.append(best.cpu().numpy() - own.cpu().numpy())
    return np.concatenate(nv), np.concatenate(ev), np.concatenate(tg).astype(np.float32)


def train_ordering_mlp(G, S, T, epochs: int = 3, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
                       max_rows: int = 2_000_000):
    """Train an OrderingMLP on plain runs over the queries (S, T)."""
    import torch
    near_v, end_v, target = collect_labels(G, S, T)
    rng = np.random.default_rng([seed, 11])
    if len(target) > max_rows:
        keep = rng.choice(len(target), max_rows, replace=False)
        near_v, end_v, target = near_v[keep], end_v[keep], target[keep]
    mean, std = float(target.mean()), float(target.std() + 1e-6)
    tnorm = ((target - mean) / std).astype(np.float32)
    model = OrderingMLP(seed=seed)
    n = len(tnorm)
    y = torch.empty(batch, dtype=torch.float32, device="cuda")
    z1 = torch.empty((batch, 256), dtype=torch.float32, device="cuda")
    work = torch.empty((batch, 256), dtype=torch.float32, device="cuda")
    grads = torch.empty(N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        ep_loss, nb = 0.0, 0
        for i in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[i:i + batch]
            va = torch.from_numpy(near_v[idx].view(np.int32)).cuda()
            vb = torch.from_numpy(end_v[idx].view(np.int32)).cuda()
            tg = torch.from_numpy(tnorm[idx]).cuda()
            b = len(idx)
            X = _mhr.mhr_mlp_features(G, va, vb)
            _mhr.mhr_mlp_forward(model, X, y[:b], z1[:b])
            _mhr.mhr_mlp_backward(model, X, tg, y[:b], z1[:b], work[:b], grads, loss)
            model.step += 1
            _mhr.mhr_mlp_adam(model.params, grads, model.m1, model.m2, lr, model.step)
            model.refresh()
            ep_loss += float(loss.item())
            nb += 1
        losses.append(ep_loss / max(nb, 1))
    model.fold_target_scale(mean, std)
    return model, TrainReport(rows=n, epochs=epochs, loss_first=losses[0], loss_last=losses[-1],
                              target_mean=mean, target_std=std)


def time_forward(rows: int = 262_144, repeat: int = 10, warmup: int = 3, seed: int = 1) -> dict:
    """CUDA-event time of the network's dense forward (TMA + tcgen05) over
    `rows` random bf16 feature rows, without the pre-activation output (the
    form the order keys use); returns microseconds per call and TFLOP/s of
    the first layer's 2 x 256 x 256 flops per row."""
    import torch
    model = OrderingMLP(seed=seed)
    g = torch.Generator(device="cuda").manual_seed(seed)
    X = torch.randn((rows, 256), generator=g, device="cuda").to(torch.bfloat16).view(torch.int16)
    y = torch.empty(rows, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        _mhr.mhr_mlp_forward(model, X, y)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(repeat):
        _mhr.mhr_mlp_forward(model, X, y)
    t1.record()
    torch.cuda.synchronize()
    us = t0.elapsed_time(t1) * 1e3 / repeat
    return {"rows": rows, "us_per_call": us, "tflops": 2.0 * 256 * 256 * rows / (us * 1e-6) / 1e12}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="time the ordering MLP's dense forward on the GPU")
    ap.add_argument("--rows", type=int, default=262_144)
    ap.add_argument("--repeat", type=int, default=10)
    a = ap.parse_args()
    print(json.dumps(time_forward(a.rows, a.repeat)))
