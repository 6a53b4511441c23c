"""Training and use of the learned warm start (``include/vbh_ws.h``).

Data sets come from the method's own generator (``synth``), shaped like the
batched workload: N cells log-uniform in [n_lo, n_hi], G genes uniform on
{48, 96} (V = N G observations), S uniform on 2..10, K_true ~ Dirichlet(alpha
1), each with its own seed.  Their CAVI fixed points, computed by the batched
form (``vbh_fit_batched``), are the targets: kappa, ln E[rho] and the Cholesky
factor of Sigma0 = W^{-1} / nu with its diagonal as logarithms, in the output
slots of vbh_ws.h, standardised per S; a data set whose fit did not converge
within the sweep cap is left out.  The encoder is trained by the library's own
tensor-core forward and backward kernels (weighted mean squared error, Adam)
on up to ``n_cap`` pooled observations per data set; predictions pool every
observation.

    python -m paper_2401_10068_gb300.warmstart --sets 8192 --out ws.npz

writes the parameters and the standardisation; ``load`` restores them.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import synth, vbh

ROWS_PER_CALL = 1 << 25            # pooled observations per encoder call (the library allows 2^26)


def shapes(count: int, seed0: int, n_lo: int, n_hi: int, s_lo: int = 2, s_hi: int = 10, genes=(48, 96)):
    """(V, S) of `count` data sets of the batched workload's shape."""
    rng = np.random.default_rng(seed0)
    N = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)
    G = rng.choice(np.asarray(genes), size=count)
    S = rng.integers(s_lo, s_hi + 1, size=count)
    return N * G, S


def make_sets(count: int, seed0: int, n_lo: int, n_hi: int, alpha: float = 0.5, device="cuda", s_lo: int = 2,
              s_hi: int = 10):
    """`count` generator data sets (device tensors) and their S."""
    V, S = shapes(count, seed0, n_lo, n_hi, s_lo, s_hi)
    rs, ds = [], []
    for b in range(count):
        r, d, _ = synth.generate_device(int(V[b]), int(S[b]), seed=seed0 * 1_000_003 + b, alpha=alpha, device=device)
        rs.append(r)
        ds.append(d)
    return rs, ds, [int(x) for x in S]


def target_from_result(res: dict, S: int):
    """The 64 output slots of a fixed point and the slots' loss weights."""
    M = S - 1
    t = np.zeros(vbh.WS_P)
    t[:M] = res["kappa"]
    t[9] = math.log(res["a_rho"] / res["b_rho"])
    sig = np.asarray(res["Winv"], dtype=np.float64).reshape(M, M) / res["nu"]
    L = np.linalg.cholesky(sig)
    for j in range(M):
        for k in range(j + 1):
            t[10 + j * (j + 1) // 2 + k] = math.log(L[j, j]) if j == k else L[j, k]
    return t, vbh.ws_slots(S).astype(np.float64)


def targets(results, Ss):
    """Targets and weights of the converged fits (weight 0 for the others)."""
    T = np.zeros((len(results), vbh.WS_P))
    W = np.zeros((len(results), vbh.WS_P))
    for b, (res, S) in enumerate(zip(results, Ss)):
        if not res["converged"]:
            continue
        T[b], W[b] = target_from_result(res, S)
    return T, W


def norm_from(T, W, Ss):
    """Per-S mean and deviation of every used slot (rows S of an 11 x 64 table)."""
    mean = np.zeros((vbh.WS_SMAX + 1, vbh.WS_P))
    std = np.ones((vbh.WS_SMAX + 1, vbh.WS_P))
    Ss = np.asarray(Ss)
    for S in range(2, vbh.WS_SMAX + 1):
        sel = (Ss == S) & (W[:, 9] > 0)
        if sel.sum() < 2:
            continue
        mean[S] = T[sel].mean(axis=0)
        std[S] = np.maximum(T[sel].std(axis=0), 1e-6)
    return mean, std


def standardise(T, W, Ss, mean, std):
    Ss = np.asarray(Ss)
    return np.where(W > 0, (T - mean[Ss]) / std[Ss], 0.0)


def train(ws: vbh.WarmStart, rs, ds, Ss, Tn, W, epochs: int, batch: int, lr: float, n_cap: int = 32768,
          seed: int = 0, log=None, lr_min: float | None = None):
    """Adam over shuffled mini-batches of data sets (sets with no used target
    are skipped), the learning rate decaying from lr to lr_min (default lr /
    20) on a cosine over the epochs; returns the mean loss per epoch."""
    import torch
    dev = rs[0].device
    keep = np.nonzero(W.sum(axis=1) > 0)[0]
    rng = np.random.default_rng(seed)
    Tt = torch.from_numpy(np.asarray(Tn, dtype=np.float32)).to(dev)
    Wt = torch.from_numpy(np.asarray(W, dtype=np.float32)).to(dev)
    losses = []
    lo = lr / 20.0 if lr_min is None else lr_min
    for ep in range(epochs):
        lr_ep = lo + 0.5 * (lr - lo) * (1.0 + math.cos(math.pi * ep / max(epochs - 1, 1)))
        perm = rng.permutation(keep)
        tot, cnt = 0.0, 0
        for s0 in range(0, len(perm) - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            it = torch.from_numpy(idx).to(dev)
            tot += ws.train_step([rs[i] for i in idx], [ds[i] for i in idx], [Ss[i] for i in idx],
                                 [n_cap] * len(idx), Tt.index_select(0, it).contiguous(),
                                 Wt.index_select(0, it).contiguous(), lr_ep)
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.5f}")
    return losses


def predict(ws: vbh.WarmStart, rs, ds, Ss, priors=None):
    """Starting points of every data set, in calls of at most ROWS_PER_CALL pooled observations."""
    out = []
    b = 0
    while b < len(rs):
        e, rows = b, 0
        while e < len(rs) and (e == b or rows + int(rs[e].shape[0]) + 128 <= ROWS_PER_CALL):
            rows += (int(rs[e].shape[0]) + 127) // 128 * 128
            e += 1
        out += ws.predict(rs[b:e], ds[b:e], Ss[b:e], None if priors is None else priors[b:e])
        b = e
    return out


def save(ws: vbh.WarmStart, path: str):
    np.savez(path, params=ws.get_params(), mean=ws.mean, std=ws.std)


def load(path: str, device: int = 0, stream=None) -> vbh.WarmStart:
    z = np.load(path)
    ws = vbh.WarmStart(device=device, stream=stream)
    ws.set_params(z["params"])
    ws.set_norm(z["mean"], z["std"])
    return ws


def fit_and_train(h: vbh.Handle, ws: vbh.WarmStart, count: int, seed0: int, n_lo: int, n_hi: int, tol: float,
                  cap: int, epochs: int, batch: int, lr: float, n_cap: int, log=None, targets_in=None,
                  s_lo: int = 2, s_hi: int = 10):
    """Generate `count` data sets, their fixed points (batched form, unless
    `targets_in` = (T, W) from an earlier run on the same seeds) and train the
    encoder on the converged ones; returns a summary with the targets."""
    t0 = time.perf_counter()
    rs, ds, Ss = make_sets(count, seed0, n_lo, n_hi, s_lo=s_lo, s_hi=s_hi)
    if targets_in is None:
        res = h.fit_batched(rs, ds, Ss, None, tol=tol, max_iter=cap)
        T, W = targets(res, Ss)
    else:
        T, W = targets_in
    t_fit = time.perf_counter() - t0
    mean, std = norm_from(T, W, Ss)
    ws.set_norm(mean, std)
    Tn = standardise(T, W, Ss, mean, std)
    t1 = time.perf_counter()
    losses = train(ws, rs, ds, Ss, Tn, W, epochs, batch, lr, n_cap, log=log)
    t_train = time.perf_counter() - t1
    conv = int((W[:, 9] > 0).sum())
    del rs, ds
    return {"sets": count, "converged": conv, "fixed_points_s": t_fit, "train_s": t_train, "losses": losses,
            "T": T, "W": W}


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=8192)
    ap.add_argument("--n-lo", type=int, default=200)
    ap.add_argument("--n-hi", type=int, default=50000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--cap", type=int, default=4000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--n-cap", type=int, default=32768)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default="ws.npz")
    args = ap.parse_args()
    stream = torch.cuda.current_stream()
    h = vbh.Handle(0, stream)
    ws = vbh.WarmStart(seed=args.seed, stream=stream)
    info = fit_and_train(h, ws, args.sets, args.seed, args.n_lo, args.n_hi, args.tol, args.cap, args.epochs,
                         args.batch, args.lr, args.n_cap, log=lambda s: print(s, flush=True))
    save(ws, args.out)
    print({k: v for k, v in info.items() if k != "losses"}, flush=True)


if __name__ == "__main__":
    main()
