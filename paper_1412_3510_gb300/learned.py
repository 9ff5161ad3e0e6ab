"""Training driver for the learned sketch weighting.

Labels come from the method itself: the plain PCA with a wider sketch
and more power iterations (Section 5's accuracy grows with both) gives V_k for
each training matrix, and rpca_leverage_target turns V_k into the log relative
leverage t_j = log(n |V_k[j, :]|^2 / k + 1e-3) that the MLP learns to predict
from the column features.  Every arithmetic step runs in librpca.so kernels;
this module only arranges the buffers and the loop.
"""
from __future__ import annotations

import math
import time

import torch

from . import _lib as L
from .rpca import (Batch, batch_col_offsets, rpca_batched_features, rpca_dense, rpca_gaussian_omega,
                   rpca_leverage_target, rpca_mlp_adam, rpca_mlp_loss_grad, rpca_mlp_pack, workspace)

F_IN, H = L.RPCA_MLP_FEATURES, L.RPCA_MLP_HIDDEN


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-style initial parameters (N(0, 2 / fan_in) weights, zero biases); the normal
    draws come from the library's Philox stream (seed, 3)."""
    z = rpca_gaussian_omega(F_IN * H + H * H + H, 1, seed, 3, device=device).view(-1)
    p = torch.zeros(L.RPCA_MLP_PARAMS, dtype=torch.float32, device=device)
    o = 0
    p[o:o + F_IN * H] = z[:F_IN * H] * math.sqrt(2.0 / F_IN); o += F_IN * H + H
    p[o:o + H * H] = z[F_IN * H:F_IN * H + H * H] * math.sqrt(2.0 / H); o += H * H + H
    p[o:o + H] = z[F_IN * H + H * H:] * math.sqrt(1.0 / H)
    return p


def leverage_dataset(mats, k: int, l_label: int | None = None, its_label: int = 4, raw: bool = False,
                     seed: int = 0):
    """(features (sum n_i) x 16, targets (sum n_i)) for a list of training matrices.

    The labelling runs use the dense entry point one matrix at a time (its sketch
    width is not bounded by the batched kernel's per-CTA buffer)."""
    ts = []
    for a in mats:
        l = min(l_label or k + 16, a.shape[0], a.shape[1])
        _, _, V = rpca_dense(a, k, l, its=its_label, raw=raw, seed=seed + 1)
        ts.append(rpca_leverage_target(V, k))
    batch = Batch(mats, k)
    offs, _ = batch_col_offsets(batch)
    F = rpca_batched_features(batch, raw=raw, seed=seed, col_offsets=offs)
    return F, torch.cat(ts)


def leverage_dataset_family(make, specs, k: int, l_label: int, its_label: int = 6, raw: bool = False,
                            seed: int = 0, chunk: int = 2048):
    """(features, targets) over a large family of matrices, generated and labelled in
    chunks: make(spec) returns one matrix on the device; each chunk is labelled by one
    batched launch (sketch width l_label, its_label power iterations) and freed before
    the next.  Matrices whose labelling run reports an error are left out.
    Returns (F, t, info)."""
    from .rpca import rpca_batched
    Fs, ts = [], []
    skipped = 0
    for c0 in range(0, len(specs), chunk):
        mats = [make(sp) for sp in specs[c0:c0 + chunk]]
        batch = Batch(mats, k)
        _, _, V = rpca_batched(batch, l=l_label, its=its_label, raw=raw, seed=seed + 1)
        offs, _ = batch_col_offsets(batch)
        F = rpca_batched_features(batch, raw=raw, seed=seed, col_offsets=offs)
        ok = (batch.status == 0).cpu().tolist()
        o = 0
        for a, v, good in zip(mats, V, ok):
            n = int(a.shape[1])
            if good:
                ts.append(rpca_leverage_target(v, k))
                Fs.append(F[o:o + n])
            else:
                skipped += 1
            o += n
        Fs = [torch.cat(Fs)]
        ts = [torch.cat(ts)]
        del mats, batch, V, F
    return Fs[0], ts[0], {"matrices": len(specs) - skipped, "skipped": skipped}


def train_mlp(F: torch.Tensor, t: torch.Tensor, steps: int = 2000, batch: int = 4096, lr: float = 1e-3,
              seed: int = 0, params: torch.Tensor | None = None, log_every: int = 0):
    """Adam on the mean squared error over shuffled minibatches.  Returns (params, info)."""
    dev = F.device
    p = init_params(seed, dev) if params is None else params.clone()
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    N = F.shape[0]
    bs = min(batch, N)
    grad = torch.empty_like(p)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    ws = workspace(int(L.load().rpca_mlp_grad_workspace_size(bs)), dev)
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    per_epoch = max(N // bs, 1)
    losses = []
    t0 = time.perf_counter()
    Fs = ts = None
    for step in range(1, steps + 1):
        e = (step - 1) % per_epoch
        if e == 0:
            perm = torch.randperm(N, generator=gen).to(dev)
            Fs = F[perm].contiguous()
            ts = t[perm].contiguous()
        sl = slice(e * bs, (e + 1) * bs)
        rpca_mlp_loss_grad(p, Fs[sl], ts[sl], grad=grad, loss=loss, ws=ws)
        rpca_mlp_adam(p, grad, m1, m2, step, lr)
        if log_every and step % log_every == 0:
            losses.append((step, float(loss.item())))
    torch.cuda.synchronize(dev)
    return p, {"steps": steps, "batch": bs, "samples": N, "seconds": time.perf_counter() - t0, "losses": losses}


def train_sketch_mlp(mats, k: int, l_label: int | None = None, its_label: int = 4, raw: bool = False,
                     steps: int = 2000, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    """Labels from the plain method, then training.  Returns (params, packed, info)."""
    t0 = time.perf_counter()
    F, t = leverage_dataset(mats, k, l_label, its_label, raw, seed)
    torch.cuda.synchronize(F.device)
    t_label = time.perf_counter() - t0
    params, info = train_mlp(F, t, steps=steps, batch=batch, lr=lr, seed=seed)
    info["label_seconds"] = t_label
    info["target_var"] = float(t.var().item())
    return params, rpca_mlp_pack(params), info


def train_sketch_mlp_family(make, specs, k: int, l_label: int, its_label: int = 6, raw: bool = False,
                            steps: int = 6000, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
                            chunk: int = 2048):
    """leverage_dataset_family, then training.  Returns (params, packed, info)."""
    t0 = time.perf_counter()
    F, t, dinfo = leverage_dataset_family(make, specs, k, l_label, its_label, raw, seed, chunk)
    torch.cuda.synchronize(F.device)
    t_label = time.perf_counter() - t0
    params, info = train_mlp(F, t, steps=steps, batch=batch, lr=lr, seed=seed)
    info |= dinfo
    info["label_seconds"] = t_label
    info["target_var"] = float(t.var().item())
    info["final_mse"] = float(rpca_mlp_loss_grad(params, F[:65536].contiguous(), t[:65536].contiguous())[0].item())
    return params, rpca_mlp_pack(params), info


def batched_learned_weights(batch: Batch, packed: torch.Tensor, raw: bool = False, seed: int = 0):
    """Per-item weight vectors d_i (views into one buffer) for rpca_batched's col_weights."""
    from .rpca import rpca_mlp_forward
    offs, total = batch_col_offsets(batch)
    F = rpca_batched_features(batch, raw=raw, seed=seed, col_offsets=offs)
    _, d = rpca_mlp_forward(packed, F, want_y=False, want_d=True)
    out, o = [], 0
    for a in batch.mats:
        n = int(a.shape[1])
        out.append(d[o:o + n])
        o += n
    return out, d
