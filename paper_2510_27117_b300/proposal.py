"""Training driver of the learned proposal (an added pattern; the paper
has no network).

Data: plain GFORS runs (p = x_k) on seeded instances; at every sampling
trigger the 8 per-variable features are read (gfors_get_features) and, once
the run ends, every recorded feature row is labelled with the incumbent's
bit for that variable.  Training: mean BCE on the logit with Adam, all
arithmetic in the library's CUDA kernels (gfors_mlp_loss_grad,
gfors_mlp_adam); torch only supplies the device buffers.
"""
from __future__ import annotations

import numpy as np

from . import gfors as G

F, H = 8, 128


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style initialisation, packed W1 b1 W2 b2 w3 b3."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, F)) * np.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3,
                           [0.0]]).astype(np.float32)


def collect(instances, prm_kw: dict, iters: int, k_int: int):
    """Plain runs; returns (features [rows x 8], labels [rows]) of every
    trigger of every instance whose run found an incumbent."""
    feats, labels = [], []
    for q, inst in enumerate(instances):
        prm = G.default_params(k_int=k_int, **prm_kw)
        h = G.load(inst, prm)
        rec = []
        rid = 0
        for _ in range(iters // k_int):
            h.pdhg_steps(k_int)
            rec.append(h.get_features(0))
            h.sample_eval(prm.k_r, rid, 0)
            rid += prm.k_r
        h.final_round()
        inc = h.incumbent(0)
        h.destroy()
        if not inc["found"]:
            continue
        y = inc["x"].astype(np.float32)
        for f in rec:
            feats.append(f)
            labels.append(y)
    return np.concatenate(feats), np.concatenate(labels)


def train(feat: np.ndarray, label: np.ndarray, epochs: int = 5, batch: int = 32768,
          lr: float = 1e-3, seed: int = 0, W0: np.ndarray | None = None):
    """Adam on mean BCE; returns (weights, per-epoch mean losses)."""
    import torch
    dev = "cuda"
    W = torch.from_numpy(init_weights(seed) if W0 is None else W0.copy()).to(dev)
    m = torch.zeros_like(W)
    v = torch.zeros_like(W)
    g = torch.zeros_like(W)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    Fd = torch.from_numpy(np.ascontiguousarray(feat, np.float32)).to(dev)
    Yd = torch.from_numpy(np.ascontiguousarray(label, np.float32)).to(dev)
    n = Fd.shape[0]
    rng = np.random.default_rng(seed)
    t = 0
    hist = []
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        tot, cnt = 0.0, 0
        for a in range(0, n, batch):
            idx = perm[a:a + batch]
            fb = Fd[idx].contiguous()
            yb = Yd[idx].contiguous()
            nb = fb.shape[0]
            G.mlp_loss_grad(W.data_ptr(), nb, fb.data_ptr(), yb.data_ptr(), g.data_ptr(),
                            loss.data_ptr())
            t += 1
            G.mlp_adam(W.numel(), W.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), t,
                       lr=lr)
            tot += float(loss.item()) * nb
            cnt += nb
        hist.append(tot / cnt)
    torch.cuda.synchronize()
    return W.cpu().numpy(), hist
