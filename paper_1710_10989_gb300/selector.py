"""Training of the (m, s)-proposing network.

    python -m paper_1710_10989_gb300.selector train [--count 1000000] [--epochs 8]

(Held-out evaluation against the paper's rule and the alpha rule, with its
accuracy check against the CPU oracle, is bench.py's learned workload.)

Training matrices: the batched workload's families (half Gaussian, half
V diag(lambda) V^-1 with cond_2(V) = 1e3, lambda ~ N(0, 4)) with N uniform on
16..512 and 1-norms log-uniform on [1e-3, 1e2]. A million such matrices are
too many to build on the host, so they are generated on the GPU in chunks of
one size (torch's seeded CUDA generator and batched QR; input generation only;
within a chunk the orthogonal factors U, W of V come from a pool of 8 each).
Per matrix the library's data mode returns the 5 features and the exact
||A^k||_1; the label is the cheapest (m, s) certified by ||A||_1 or by
alpha_2 = max(||A^2||^(1/2), ||A^3||^(1/3)) (bbc_select_certified). The network
(5 -> 64 -> 64 -> 60, classes = degree index * 10 + s) is trained with the
library's own forward/backward/Adam kernels and saved to selector_weights.npz.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
WEIGHTS = os.path.join(HERE, "selector_weights.npz")
S_VALUES = 10
HIDDEN = 64
DEGREES = (1, 2, 4, 8, 12, 18)


def gpu_matrices(torch, n: int, count: int, gen, norm_lo=1e-3, norm_hi=1e2, kinds=None):
    """`count` matrices of size n on the GPU (float64): even slots Gaussian, odd
    slots V diag(lambda) V^-1 with cond_2(V) = 1e3; 1-norms log-uniform."""
    dev = "cuda"
    A = torch.randn((count, n, n), generator=gen, device=dev, dtype=torch.float64) / n ** 0.5
    odd = torch.arange(count, device=dev) % 2 == 1 if kinds is None else kinds
    k = int(odd.sum())
    if k:
        # a pool of orthogonal factors (QR of Gaussians, sign-fixed) per chunk; each
        # matrix pairs one U with one W, so V = U S W^T keeps cond_2(V) = 1e3
        pool = min(8, k)

        def orth():
            Q, R = torch.linalg.qr(torch.randn((pool, n, n), generator=gen, device=dev, dtype=torch.float64))
            return Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2)).unsqueeze(1)
        Up, Wp = orth(), orth()
        ia = torch.randint(0, pool, (k,), generator=gen, device=dev)
        ib = torch.randint(0, pool, (k,), generator=gen, device=dev)
        U, Wm = Up[ia], Wp[ib]
        sv = torch.logspace(0.0, -3.0, n, device=dev, dtype=torch.float64)
        lam = torch.randn((k, n), generator=gen, device=dev, dtype=torch.float64) * 2.0
        V = (U * sv) @ Wm.transpose(1, 2)
        Vinv = (Wm / sv) @ U.transpose(1, 2)
        A[odd] = (V * lam.unsqueeze(1)) @ Vinv
    target = torch.exp(torch.empty(count, device=dev, dtype=torch.float64).uniform_(
        np.log(norm_lo), np.log(norm_hi), generator=gen))
    cur = A.abs().sum(dim=1).max(dim=1).values
    return A * (target / cur).view(-1, 1, 1)


def make_dataset(count: int, seed: int, chunk: int = 256, log_every: int = 200):
    import torch

    from paper_1710_10989_gb300 import api
    h = api.Handle(0)
    h.batch_reserve(512)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    feats, norms, sizes = [], [], []
    done, t0 = 0, time.time()
    while done < count:
        c = min(chunk, count - done)
        n = int(rng.integers(16, 513))
        A = gpu_matrices(torch, n, c, gen)
        b = api.Batch(list(A.unbind(0)))
        f, nr = h.selector_data(b)
        feats.append(f.cpu().numpy())
        norms.append(nr.cpu().numpy())
        sizes.append(np.full(c, n))
        done += c
        if len(feats) % log_every == 0:
            print(f"  {done}/{count} matrices, {time.time() - t0:.0f} s", flush=True)
    h.close()
    return np.concatenate(feats), np.concatenate(norms), np.concatenate(sizes)


def labels_of(norms, u=2.0 ** -53):
    from paper_1710_10989_gb300 import api
    out = np.empty(len(norms), dtype=np.int64)
    for i, nr in enumerate(norms):
        m, s = api.select_certified(nr[:3], u)
        out[i] = DEGREES.index(m) * S_VALUES + min(s, S_VALUES - 1)
    return out


def plain_class(norms, u=2.0 ** -53):
    from paper_1710_10989_gb300 import api
    out = np.empty(len(norms), dtype=np.int64)
    for i, nr in enumerate(norms):
        m, s = api.select(float(nr[0]), u)
        out[i] = DEGREES.index(m) * S_VALUES + min(s, S_VALUES - 1)
    return out


def cost_of(cls):
    """products + s of each class (Table 3: degree index i costs i products)."""
    cls = np.asarray(cls)
    return cls // S_VALUES + cls % S_VALUES


def train(args):
    import torch

    from paper_1710_10989_gb300 import api
    t0 = time.time()
    X, norms, sizes = make_dataset(args.count, args.seed)
    ok = np.isfinite(X).all(1) & np.isfinite(norms[:, :3]).all(1)
    X, norms, sizes = X[ok], norms[ok], sizes[ok]
    y = labels_of(norms)
    t_data = time.time() - t0
    mu, sd = X.mean(0), X.std(0) + 1e-6
    net = api.MLP(5, HIDDEN, 6 * S_VALUES, seed=args.seed)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    Xn = (Xd - torch.from_numpy(mu).cuda()) / torch.from_numpy(sd).cuda()
    n = len(X)
    perm_gen = torch.Generator(device="cuda").manual_seed(args.seed + 1)
    steps = 0
    t1 = time.time()
    for ep in range(args.epochs):
        perm = torch.randperm(n, generator=perm_gen, device="cuda")
        lr = args.lr * (0.5 ** (ep // 3))
        for i in range(0, n, args.batch):
            idx = perm[i:i + args.batch]
            net.train_step(Xn[idx], yd[idx], lr=lr)
            steps += 1
        with torch.no_grad():
            pred = torch.cat([net.forward(Xn[i:i + 65536]).argmax(1) for i in range(0, n, 65536)])
            acc = float((pred == yd).float().mean())
        print(f"epoch {ep}: train accuracy {acc:.4f}", flush=True)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    meta = {"count": int(n), "seed": args.seed, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
            "train_accuracy": acc, "steps": steps, "data_seconds": t_data, "train_seconds": t_train,
            "label": "cheapest (m, s) certified by ||A||_1 or alpha_2 (u = 2^-53)", "S": S_VALUES,
            "hidden": HIDDEN, "mean_label_cost": float(cost_of(y).mean()),
            "mean_plain_cost": float(cost_of(plain_class(norms[:20000])).mean())}
    np.savez(args.out, params=net.params.cpu().numpy(), mu=mu.astype(np.float32), sd=sd.astype(np.float32),
             meta=json.dumps(meta))
    print(json.dumps(meta), flush=True)


def load(path=WEIGHTS):
    d = np.load(path)
    return d["params"], d["mu"], d["sd"], json.loads(str(d["meta"]))


def install(h, path=WEIGHTS):
    from paper_1710_10989_gb300 import api
    params, mu, sd, meta = load(path)
    net = api.MLP(5, meta["hidden"], 6 * meta["S"], params=params)
    h.batch_set_selector(net, meta["S"], mu, sd)
    return net, meta


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=("train",))
    ap.add_argument("--count", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args()
    a.count = a.count or 1_000_000
    a.seed = a.seed or 11
    train(a)


if __name__ == "__main__":
    main()
