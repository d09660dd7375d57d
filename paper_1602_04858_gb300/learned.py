"""Learned initial guess for the V-cycle-preconditioned GMRES (RT_0, 2-D).

Data: seeded problems on n x n cells (lognormal c = exp(G), G ~ GRF(sigma,
ell); body force f ~ GRF(1, n/8) per component; no divergence source,
no-slip walls), solved by the method itself (mg_solve, FP32 V-cycle inside
FP64 FGMRES, tight tolerance).  The network (mg_cnn_*) learns the per-cell
solution from (log c, f); a solve started from its guess must still reach
the same residual tolerance as one started from zero.

    python -m paper_1602_04858_gb300.learned --n 128 --train 2000 --test 200 --out weights.npz

Everything numerical runs in the CUDA library; this module orders the calls
and keeps the data set on the device.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, mgdarcy


def problem(seed: int, n: int, sigma: float = 2.0, ell: float = 8.0):
    """Coefficient c (n, n) and body force f (2, n, n) of one seeded problem."""
    c = inputs.lognormal_c(n, 2, sigma, ell, seed)
    f = np.stack([inputs.grf(n, 2, 1.0, n / 8.0, 1_000_000 + 2 * seed),
                  inputs.grf(n, 2, 1.0, n / 8.0, 1_000_001 + 2 * seed)])
    return c, f


def hierarchy_args(n: int):
    """Levels 4x4 -> n x n; the sub-cycle three levels below the finest is folded
    (dense operator of at most a few tens of MB, cheap to set up per problem)."""
    n_coarse = 4
    levels = int(np.log2(n // n_coarse)) + 1
    return dict(dim=2, n_coarse=n_coarse, n_levels=levels, degree=0, mu=0.01, dense_level=max(0, levels - 4))


def solve_problem(torch, seed, n, x0_fn=None, tol=1e-8, maxit=200, precision="fp32", smooth_steps=1):
    """Sets up and solves one problem; returns (stats, x, c_dev, f_dev, setup_ms).

    With x0_fn the solve starts from its guess after `smooth_steps` symmetric
    Schwarz smoothing steps on the finest level (each about 1/8 of a variable
    V-cycle with m(J) = 2): the network is accurate in the smooth part of the
    solution, the smoother removes the rest.
    """
    c, f = problem(seed, n)
    cd = torch.as_tensor(c, device="cuda")
    fd = torch.as_tensor(f.reshape(2, -1), device="cuda").contiguous()
    a = hierarchy_args(n)
    t0 = time.perf_counter()
    G = mgdarcy.Multigrid(a["dim"], a["n_coarse"], a["n_levels"], a["degree"], a["mu"], cd,
                          precision=precision, dense_level=a["dense_level"])
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    nu, np_ = G.sizes()
    b = torch.zeros(nu + np_, dtype=torch.float64, device="cuda")
    G.load_vector(fd, None, b)
    x = torch.zeros_like(b)
    use_x0 = False
    if x0_fn is not None:
        x0_fn(cd, fd, x)
        if smooth_steps > 0:
            G.smooth(a["n_levels"] - 1, x, b, steps=smooth_steps)
        use_x0 = True
    st, status = G.solve(b[:nu].contiguous(), b[nu:].contiguous(), x, use_x0=use_x0, tol=tol, maxit=maxit,
                         check=False)
    return st, x, cd, fd, setup_ms


def build_dataset(torch, net, seeds, n, tol=1e-10, log=None):
    """Solves the seeded problems; returns their (c, f, x) on the device."""
    data = []
    t0 = time.perf_counter()
    for k, s in enumerate(seeds):
        st, x, cd, fd, _ = solve_problem(torch, s, n, tol=tol, maxit=400)
        data.append((cd, fd, x))
        if log and (k + 1) % 250 == 0:
            log(f"{k + 1} solves, {time.perf_counter() - t0:.1f} s")
    torch.cuda.synchronize()
    return data


def fit_normalisation(torch, net, data):
    """Per-channel mean and standard deviation of the raw features and targets
    (network normalisation set to the identity while they are formed)."""
    n = net.n
    net.set_normalisation(np.zeros(3), np.ones(3), np.zeros(3), np.ones(3))
    buf = torch.zeros((2, 3, n * n), dtype=torch.float32, device="cuda")
    s1 = np.zeros((2, 3))
    s2 = np.zeros((2, 3))
    for cd, fd, x in data:
        net.features(cd, fd, buf[0])
        net.targets(x, buf[1])
        h = buf.cpu().numpy().astype(np.float64)
        s1 += h.sum(axis=2)
        s2 += (h * h).sum(axis=2)
    cnt = len(data) * n * n
    mean = s1 / cnt
    std = np.sqrt(np.maximum(s2 / cnt - mean * mean, 0.0)) + 1e-12
    return mean[0], std[0], mean[1], std[1]


def normalised_tensors(torch, net, data):
    """Normalised features and targets of the data set, formed by the library kernels."""
    n = net.n
    feats = torch.zeros((len(data), 3, n * n), dtype=torch.float32, device="cuda")
    targs = torch.zeros((len(data), 3, n * n), dtype=torch.float32, device="cuda")
    for k, (cd, fd, x) in enumerate(data):
        net.features(cd, fd, feats[k])
        net.targets(x, targs[k])
    torch.cuda.synchronize()
    return feats, targs


def train(torch, net, feats, targs, epochs=30, batch=16, lr=2e-3, seed=0, log=None):
    """Adam on minibatches of the (normalised) data set; returns the loss history."""
    g = np.random.default_rng(seed)
    n_samples = feats.shape[0]
    hist = []
    for ep in range(epochs):
        order = g.permutation(n_samples)
        tot, cnt = 0.0, 0
        for s in range(0, n_samples - batch + 1, batch):
            idx = torch.as_tensor(order[s:s + batch], device="cuda")
            xb = feats.index_select(0, idx).contiguous()
            yb = targs.index_select(0, idx).contiguous()
            tot += net.train_step(xb, yb, batch, lr)
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def evaluate(torch, net, seeds, n, tol=1e-8, smooth_steps=1, fp64=False):
    """Iterations and solve time from the zero and from the (smoothed) learned
    guess (FP32 V-cycle in FP64 FGMRES), and with fp64 the plain FP64 solve
    from zero beside them."""
    rows = []
    for s in seeds:
        st0, _, _, _, _ = solve_problem(torch, s, n, tol=tol)
        st1, _, _, _, _ = solve_problem(torch, s, n, x0_fn=lambda c, f, x: net.guess(c, f, x), tol=tol,
                                        smooth_steps=smooth_steps)
        row = dict(seed=s, zero_its=st0.iterations, zero_ms=st0.solve_ms, zero_conv=st0.converged,
                   learned_its=st1.iterations, learned_ms=st1.solve_ms, learned_conv=st1.converged,
                   learned_initial_rel_residual=st1.initial_rel_residual)
        if fp64:
            st2, _, _, _, _ = solve_problem(torch, s, n, tol=tol, precision="fp64")
            row.update(fp64_its=st2.iterations, fp64_ms=st2.solve_ms, fp64_conv=st2.converged)
        rows.append(row)
    return rows


def summarise(rows):
    z = np.array([r["zero_its"] for r in rows])
    l = np.array([r["learned_its"] for r in rows])
    zt = np.array([r["zero_ms"] for r in rows])
    lt = np.array([r["learned_ms"] for r in rows])
    return dict(problems=len(rows), zero_its_mean=float(z.mean()), learned_its_mean=float(l.mean()),
                zero_its_median=float(np.median(z)), learned_its_median=float(np.median(l)),
                zero_its_max=int(z.max()), learned_its_max=int(l.max()),
                zero_ms_mean=float(zt.mean()), learned_ms_mean=float(lt.mean()),
                all_converged=bool(all(r["zero_conv"] and r["learned_conv"] and r.get("fp64_conv", True)
                                       for r in rows)),
                learned_initial_rel_residual_mean=float(np.mean([r["learned_initial_rel_residual"] for r in rows])),
                fp64_its_mean=float(np.mean([r["fp64_its"] for r in rows])) if "fp64_its" in rows[0] else None,
                fp64_ms_mean=float(np.mean([r["fp64_ms"] for r in rows])) if "fp64_ms" in rows[0] else None)


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    net = mgdarcy.CNN(args.n, max_batch=16, seed=1)
    t0 = time.perf_counter()
    data = build_dataset(torch, net, list(range(args.train)), args.n, log=lambda m: print(m, flush=True))
    gen_s = time.perf_counter() - t0
    fm, fs, tm, ts = fit_normalisation(torch, net, data)
    net.set_normalisation(fm, fs, tm, ts)
    feats, targs = normalised_tensors(torch, net, data)
    t0 = time.perf_counter()
    hist = train(torch, net, feats, targs, epochs=args.epochs, log=lambda m: print(m, flush=True))
    train_s = time.perf_counter() - t0
    rows = evaluate(torch, net, list(range(100000, 100000 + args.test)), args.n, fp64=True)
    summary = summarise(rows)
    summary.update(n=args.n, train_samples=args.train, data_generation_s=gen_s, training_s=train_s,
                   final_loss=hist[-1])
    print(json.dumps(summary))
    if args.out:
        np.savez(args.out, params=net.get_params(), norm=np.concatenate([fm, fs, tm, ts]))


if __name__ == "__main__":
    main()
