"""Host-side driver of the learned correlation surrogate: labelled pairs from
the exact Gram kernel, a training loop over the library's forward, backward
and Adam kernels, checkpoints, and the evaluation that compares surrogate,
closed form and exact Gram on modified-ZF sum rate.

Every step of the surrogate itself (labels, features, training, inference)
runs in libxlmimo; this module orders the calls, keeps the buffers and draws
minibatch orders.  The error metrics of `compare` are plain torch reductions
on the device: they judge the surrogate and are not part of it.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import inputs
from . import xlmimo as X


def label_pairs(n, freq, users, prec=X.BF16X3, model=X.FSPL_USW, weights=False, base=X.APERTURE_NONE,
                device="cuda"):
    """Features and targets of every pair of every trial (trial t: n[t]
    elements, carrier freq[t], users[t] [K][2]); trials are labelled one by one
    because each has its own array.  Returns (feat [R][6], target [R][2],
    weight [R] or None) on the device."""
    feats, targets, wts = [], [], []
    K = users.shape[1]
    ud = torch.from_numpy(np.ascontiguousarray(users)).to(device)
    for t in range(len(n)):
        lam = inputs.wavelength(float(freq[t]))
        arr = X.array(int(n[t]), lam, model=model)
        u = ud[t:t + 1]
        g = X.xlmimo_channel_gram(arr, u, prec)
        gc = X.xlmimo_corr_closed_form(arr, u)
        f, tg, w = X.xlmimo_pair_features(arr, u, g, gc, weights=weights, base=base)
        feats.append(f)
        targets.append(tg)
        if weights:
            wts.append(w)
    feat = torch.cat(feats)
    target = torch.cat(targets)
    return feat, target, (torch.cat(wts) if weights else None)


class Trainer:
    """Adam training of the network on (feat, target[, weight]) rows with a
    cosine learning-rate schedule; minibatches are contiguous slices of a
    per-epoch permutation."""

    def __init__(self, params: torch.Tensor, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
        self.params = params
        dev = params.device
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grad = torch.empty_like(params)
        self.batch = int(batch)
        self.lr = float(lr)
        self.step = 0
        self.gen = torch.Generator(device=dev).manual_seed(int(seed))
        self.out = torch.empty((self.batch, X.MLP_OUT), dtype=torch.float32, device=dev)
        self.cache = torch.empty((self.batch * X.MLP_CACHE_PER_ROW,), dtype=torch.float32, device=dev)
        self.work = torch.empty((X.xlmimo_mlp_work_floats(self.batch),), dtype=torch.float32, device=dev)
        self.loss = torch.empty((1,), dtype=torch.float32, device=dev)

    def fit(self, feat, target, weight=None, steps: int = 3000, log_every: int = 0):
        """Runs `steps` Adam steps; returns the list of (step, loss) logged."""
        R = feat.shape[0]
        if R < self.batch:
            raise ValueError(f"need at least {self.batch} rows, got {R}")
        per_epoch = R // self.batch
        perm, pos = None, per_epoch
        total = self.step + steps
        log = []
        for _ in range(steps):
            if pos == per_epoch:
                perm = torch.randperm(R, generator=self.gen, device=feat.device)
                pos = 0
            idx = perm[pos * self.batch:(pos + 1) * self.batch]
            pos += 1
            x = feat.index_select(0, idx)
            tg = target.index_select(0, idx)
            w = weight.index_select(0, idx) if weight is not None else None
            self.step += 1
            lr = 0.5 * self.lr * (1.0 + math.cos(math.pi * (self.step - 1) / max(1, total)))
            X.xlmimo_mlp_train_step(self.params, self.m, self.v, self.grad, self.step, lr, x, tg, w, self.out,
                                    self.cache, self.work, self.loss)
            if log_every and (self.step % log_every == 0 or self.step == total):
                log.append((self.step, float(self.loss.item())))
        return log

    def state(self) -> dict:
        return {"params": self.params.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(),
                "step": self.step, "rng": self.gen.get_state().cpu().numpy()}

    def save(self, path: str):
        np.savez(path, **self.state())

    def load(self, path: str):
        d = np.load(path)
        dev = self.params.device
        self.params.copy_(torch.from_numpy(d["params"]).to(dev))
        self.m.copy_(torch.from_numpy(d["m"]).to(dev))
        self.v.copy_(torch.from_numpy(d["v"]).to(dev))
        self.step = int(d["step"])
        self.gen.set_state(torch.from_numpy(d["rng"]))


def compare(arr, users, packed, snr_db=10.0, prec=X.BF16X3, scheme=X.ZF, base=X.APERTURE_NONE):
    """Exact, closed-form (paper; aperture mask; Fresnel factor) and surrogate
    Gram of the same trials and the sum rates of the receiver built on each,
    all judged on the exact channel.  Returns a dict of per-trial numpy arrays:
    rate_{exact,cf,mask,fresnel,sur}, status_*, gram_err_{cf,mask,fresnel,sur}
    (RMS over pairs of |G^_ij - G_ij| / sqrt(G_ii G_jj))."""
    B, K = users.shape[0], users.shape[1]
    g = X.xlmimo_channel_gram(arr, users, prec)
    gc = X.xlmimo_corr_closed_form(arr, users)
    gm = X.xlmimo_corr_closed_form_aperture(arr, users, X.APERTURE_MASK)
    gf = X.xlmimo_corr_closed_form_aperture(arr, users, X.APERTURE_FRESNEL)
    gs = X.xlmimo_surrogate_gram(arr, users, packed, base=base)
    power = torch.full((B, K), 10.0 ** (snr_db / 10.0), dtype=torch.float64, device=users.device)
    noise = torch.ones((B,), dtype=torch.float64, device=users.device)
    out = {}
    for name, gfil, gt in (("exact", g, None), ("cf", gc, g), ("mask", gm, g), ("fresnel", gf, g), ("sur", gs, g)):
        sinr, status, _ = X.xlmimo_beamform(gfil, power, noise, scheme, X.POWER_RXSNR, gram_true=gt)
        out["rate_" + name] = X.xlmimo_sumrate(sinr)[0].cpu().numpy()
        out["status_" + name] = status.cpu().numpy()
    d = torch.diagonal(g, dim1=1, dim2=2).real
    nrm = torch.sqrt(d[:, :, None] * d[:, None, :])
    off = ~torch.eye(K, dtype=torch.bool, device=users.device)
    for name, gh in (("cf", gc), ("mask", gm), ("fresnel", gf), ("sur", gs)):
        e = ((gh - g).abs() / nrm)[:, off]
        out["gram_err_" + name] = torch.sqrt((e ** 2).mean(dim=1)).cpu().numpy()
    return out


def main(argv=None):
    """Command line: `train` labels pairs, trains and saves a checkpoint;
    `infer` runs the fused inference on one batch (weights from a checkpoint,
    or the seeded initial ones) and prints its time."""
    import argparse
    import time

    ap = argparse.ArgumentParser(prog="python -m paper_2503_18118_gb300.surrogate")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--pairs", type=float, default=1e7)
    t.add_argument("--k", type=int, default=64)
    t.add_argument("--steps", type=int, default=8000)
    t.add_argument("--batch", type=int, default=16384)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--seed", type=int, default=5)
    t.add_argument("--base", type=int, default=0, help="aperture factor the network corrects (0 none, 1 mask, 2 Fresnel)")
    t.add_argument("--out", required=True)
    i = sub.add_parser("infer")
    i.add_argument("--checkpoint")
    i.add_argument("--trials", type=int, default=300)
    i.add_argument("--k", type=int, default=64)
    i.add_argument("--n", type=int, default=262144)
    i.add_argument("--freq-ghz", type=float, default=100.0)
    i.add_argument("--repeat", type=int, default=2)
    i.add_argument("--seed", type=int, default=6)
    i.add_argument("--base", type=int, default=0)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        trials = int(math.ceil(a.pairs / (a.k * (a.k - 1) // 2)))
        n, freq, users = inputs.surrogate_trials(a.seed, trials, a.k)
        feat, target, _ = label_pairs(n, freq, users, base=a.base)
        tr = Trainer(torch.from_numpy(inputs.mlp_init_params(a.seed)).cuda(), batch=a.batch, lr=a.lr, seed=a.seed)
        t0 = time.perf_counter()
        log = tr.fit(feat, target, steps=a.steps, log_every=max(1, a.steps // 10))
        torch.cuda.synchronize()
        for s, l in log:
            print(f"step {s} loss {l:.6g}")
        print(f"trained {a.steps} steps on {feat.shape[0]} pairs in {time.perf_counter() - t0:.2f} s")
        tr.save(a.out)
    else:
        params = torch.from_numpy(inputs.mlp_init_params(a.seed)).cuda()
        if a.checkpoint:
            params.copy_(torch.from_numpy(np.load(a.checkpoint)["params"]).cuda())
        packed = X.xlmimo_mlp_pack(params)
        arr = X.array(a.n, inputs.wavelength(a.freq_ghz * 1e9))
        r = (3.0, 30.0) if a.freq_ghz >= 60 else (5.0, 50.0)
        u = torch.from_numpy(inputs.users_polar(a.seed, a.trials, a.k, r)).cuda()
        g = torch.empty((a.trials, a.k, a.k), dtype=torch.complex128, device="cuda")
        for _ in range(a.repeat):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            X.xlmimo_surrogate_gram(arr, u, packed, g, base=a.base)
            e1.record()
            torch.cuda.synchronize()
            print(f"surrogate Gram of {a.trials} trials (K={a.k}, N={a.n}): {e0.elapsed_time(e1):.3f} ms, "
                  f"finite {bool(torch.isfinite(g).all())}")


if __name__ == "__main__":
    main()
