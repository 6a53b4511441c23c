"""Training and use of the learned warm start (``include/vbh_ws.h``).

Data sets come from the method's own generator (``synth``): for data set b,
K_true ~ Dirichlet(alpha 1) with its own seed, V_b observations.  Their CAVI
fixed points, computed by the batched form (``vbh_fit_batched``), are the
targets: kappa, ln E[rho] and the Cholesky factor of Sigma0 = W^{-1} / nu with
its diagonal as logarithms.  The encoder sees the features of n evenly spaced
observations of each data set and is trained by the library's own forward and
backward kernels (mean squared error of standardised targets, Adam).

    python -m paper_2401_10068_gb300.warmstart --S 3 --sets 20000 --out ws_s3.npz

writes the parameters and the standardisation; ``load`` restores them.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import synth, vbh


def target_from_result(res: dict, M: int) -> np.ndarray:
    """kappa, ln E[rho], packed Cholesky of Sigma0 (diagonal as logs)."""
    sig = np.asarray(res["Winv"], dtype=np.float64).reshape(M, M) / res["nu"]
    L = np.linalg.cholesky(sig)
    chol = [math.log(L[j, k]) if j == k else L[j, k] for j in range(M) for k in range(j + 1)]
    return np.concatenate([np.asarray(res["kappa"], dtype=np.float64), [math.log(res["rho_mean"])], chol])


def make_sets(S: int, count: int, seed0: int, v_lo: int, v_hi: int, alpha: float = 1.0, device="cuda"):
    """`count` data sets with V log-uniform in [v_lo, v_hi] (device tensors)."""
    rng = np.random.default_rng(seed0)
    V = np.floor(np.exp(rng.uniform(math.log(v_lo), math.log(v_hi), size=count))).astype(np.int64)
    rs, ds = [], []
    for b in range(count):
        r, d, _ = synth.generate_device(int(V[b]), S, seed=seed0 * 1_000_003 + b, alpha=alpha, device=device)
        rs.append(r)
        ds.append(d)
    return rs, ds


def fixed_points(h: vbh.Handle, rs, ds, S: int, tol: float = 1e-8, cap: int = 2000, init_states=None):
    """CAVI fits of every data set by the batched form."""
    return h.fit_batched(rs, ds, [S] * len(rs), None, tol=tol, max_iter=cap, init_states=init_states)


def build_training_set(ws: vbh.WarmStart, h: vbh.Handle, rs, ds, S: int, n: int, tol=1e-8, cap=2000):
    """Features (sets x n x F, device) and standardised targets (sets x P)."""
    import torch
    M = S - 1
    res = fixed_points(h, rs, ds, S, tol, cap)
    T = np.stack([target_from_result(x, M) for x in res])
    X = torch.empty((len(rs), n, ws.F), dtype=torch.float32, device=rs[0].device)
    for b in range(len(rs)):
        ws.features(rs[b], ds[b], n, X[b])
    mean = T.mean(axis=0)
    std = T.std(axis=0)
    std[std < 1e-6] = 1e-6
    ws.set_norm(mean, std)
    Tn = torch.from_numpy(((T - mean) / std).astype(np.float32)).to(rs[0].device)
    return X, Tn, res


def train(ws: vbh.WarmStart, X, Tn, epochs: int, batch: int, lr: float, seed: int = 0, log=None):
    """Adam over shuffled mini-batches of sets; returns the loss per epoch."""
    import torch
    nsets, n = X.shape[0], X.shape[1]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(nsets)).to(X.device)
        tot, cnt = 0.0, 0
        for s0 in range(0, nsets - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            xb = X.index_select(0, idx).contiguous()
            tb = Tn.index_select(0, idx).contiguous()
            tot += ws.train_step(xb, tb, batch, n, lr)
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.5f}")
    return losses


def save(ws: vbh.WarmStart, path: str, hidden: int):
    np.savez(path, S=ws.S, hidden=hidden, params=ws.get_params(), mean=ws.mean, std=ws.std)


def load(path: str, device: int = 0, stream=None) -> vbh.WarmStart:
    z = np.load(path)
    ws = vbh.WarmStart(int(z["S"]), int(z["hidden"]), device=device, stream=stream)
    ws.set_params(z["params"])
    ws.set_norm(z["mean"], z["std"])
    return ws


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--S", type=int, default=3)
    ap.add_argument("--hidden", type=int, default=256)
    ap.add_argument("--sets", type=int, default=20000)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--v-lo", type=int, default=9600)
    ap.add_argument("--v-hi", type=int, default=200000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default="ws.npz")
    args = ap.parse_args()
    stream = torch.cuda.current_stream()
    h = vbh.Handle(0, stream)
    ws = vbh.WarmStart(args.S, args.hidden, seed=args.seed, stream=stream)
    t0 = time.perf_counter()
    X_all, T_all = [], []
    chunk = 4096
    for c0 in range(0, args.sets, chunk):
        rs, ds = make_sets(args.S, min(chunk, args.sets - c0), args.seed + c0, args.v_lo, args.v_hi)
        res = fixed_points(h, rs, ds, args.S)
        T_all.append(np.stack([target_from_result(x, args.S - 1) for x in res]))
        X = torch.empty((len(rs), args.n, ws.F), dtype=torch.float32, device="cuda")
        for b in range(len(rs)):
            ws.features(rs[b], ds[b], args.n, X[b])
        X_all.append(X)
        del rs, ds
    X = torch.cat(X_all)
    T = np.concatenate(T_all)
    mean, std = T.mean(axis=0), np.maximum(T.std(axis=0), 1e-6)
    ws.set_norm(mean, std)
    Tn = torch.from_numpy(((T - mean) / std).astype(np.float32)).cuda()
    print(f"{len(T)} data sets and fixed points in {time.perf_counter() - t0:.1f} s", flush=True)
    train(ws, X, Tn, args.epochs, args.batch, args.lr, seed=args.seed, log=lambda s: print(s, flush=True))
    save(ws, args.out, args.hidden)
    print(f"saved {args.out} after {time.perf_counter() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main()
