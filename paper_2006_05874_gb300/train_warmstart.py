"""Train the warm-start network on the GPU and write its parameter file.

    python -m paper_2006_05874_gb300.train_warmstart --out warmstart_weights.json

1. Draw problems from ``problems.sampled_ridge`` (seeds 1000.. for training,
   900000.. held out), compute their 11 features with ``ihs_probe_features``,
   and label each with log2 of the sketch size a cold solve (m_init = 1,
   SRHT, gradient-IHS variant) settles at.
2. Fix the feature normalisation (mean and standard deviation of the training
   features) and fit the network by Adam on the mean squared error, minibatches
   of 256 (the last quarter of the steps at a tenth of the rate), every step
   one ``ihs_mlp_train_step`` launch.
3. Report the held-out error and, on the held-out problems, the cold and the
   warm-started solves side by side (wall time including the probe, gradient
   passes, levels drawn), and store all of it with the parameters.
"""
import argparse
import json
import math
import time

import numpy as np


def _label(ctx, A, b, nu):
    import torch

    d = A.shape[1]
    ctx.set_params(m_init=1)
    x = torch.zeros(d, device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.solve(A, b, nu, x)
    torch.cuda.synchronize()
    return rep, time.perf_counter() - t0, x


def build_set(ctx, seeds, log=print):
    """Features and labels of the problems drawn from `seeds`."""
    import torch

    from . import ihs
    from .problems import sampled_ridge

    feats, labels, rows = [], [], []
    f = torch.zeros(11, device="cuda", dtype=torch.float32)
    for s in seeds:
        A, b, nu, meta = sampled_ridge(s, "cuda")
        ctx.probe_features(A, nu, ctx.params.seed, f)
        try:
            rep, secs, _ = _label(ctx, A, b, nu)
        except ihs.IHSError as e:
            log("seed %d skipped: %s" % (s, e))
            continue
        feats.append(f.cpu().numpy().copy())
        labels.append(math.log2(rep.m_final))
        rows.append(dict(meta, nu=nu, m_final=int(rep.m_final), cold_s=secs, cold_passes=int(rep.grad_passes),
                         cold_levels=int(rep.n_levels), status=int(rep.status)))
        del A, b
        if len(rows) % 2000 == 0:
            log("labelled %d" % len(rows))
    log("labelled %d problems" % len(rows))
    return (np.array(feats, dtype=np.float32), np.array(labels, dtype=np.float32), rows,
            [r["seed"] for r in rows])


def _layout():
    nf, nh = 11, 64
    sizes = [("mu", nf), ("sd", nf), ("W1", nh * nf), ("b1", nh), ("W2", nh * nh), ("b2", nh), ("w3", nh),
             ("b3", 1)]
    off, o = {}, 0
    for k, s in sizes:
        off[k] = (o, s)
        o += s
    return off, o


def initial_params(X, y, seed):
    """Feature normalisation from the training set; weights N(0, 1/fan_in); b3 = mean label."""
    off, total = _layout()
    rng = np.random.default_rng(seed)
    p = np.zeros(total, dtype=np.float64)
    mu, sd = X.mean(axis=0), X.std(axis=0)
    sd = np.where(sd > 1e-3, sd, 1.0)
    p[off["mu"][0]:off["mu"][0] + 11] = mu
    p[off["sd"][0]:off["sd"][0] + 11] = sd
    for k, fan in (("W1", 11), ("W2", 64), ("w3", 64)):
        o, s = off[k]
        p[o:o + s] = rng.standard_normal(s) / math.sqrt(fan)
    p[off["b3"][0]] = float(np.mean(y))
    return p.astype(np.float32)


def train(ctx, X, y, steps, lr, batch, seed, log=print):
    import torch

    p0 = initial_params(X, y, seed)
    params = torch.as_tensor(p0, device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    Xd = torch.as_tensor(X, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    rng = np.random.default_rng(seed + 1)
    n = X.shape[0]
    hist = []
    for step in range(1, steps + 1):
        if n <= batch:
            xb, yb = Xd, yd
        else:
            idx = torch.as_tensor(rng.choice(n, batch, replace=False), device="cuda")
            xb, yb = Xd[idx].contiguous(), yd[idx].contiguous()
        want = step % 500 == 0 or step == 1
        # the last quarter of the steps runs at a tenth of the rate
        lr_t = lr if step <= 0.75 * steps else 0.1 * lr
        loss = ctx.mlp_train_step(params, m, v, step, xb, yb, lr_t, want_loss=want)
        if want:
            hist.append((step, loss))
            log("step %5d  minibatch mse %.4f" % (step, loss))
    return params, hist


def predict(ctx, params, X):
    import torch

    Xd = torch.as_tensor(X, device="cuda")
    out = torch.zeros(X.shape[0], device="cuda", dtype=torch.float32)
    ctx.mlp_forward(params, Xd, out)
    return out.cpu().numpy()


def compare_heldout(ctx, params, seeds, rows):
    """Cold vs warm-started solves on the held-out problems."""
    import torch

    from .problems import sampled_ridge

    out = []
    for s, row in zip(seeds, rows):
        A, b, nu, meta = sampled_ridge(s, "cuda")
        # one untimed cold solve so both timed runs see warm caches and a sized arena
        _label(ctx, A, b, nu)
        rep_c, t_c, xc = _label(ctx, A, b, nu)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m0, pred = ctx.warm_start(params, A, nu)
        ctx.set_params(m_init=m0)
        x = torch.zeros(A.shape[1], device="cuda", dtype=torch.float32)
        rep_w = ctx.solve(A, b, nu, x)
        torch.cuda.synchronize()
        t_w = time.perf_counter() - t0
        ctx.set_params(m_init=1)
        out.append(dict(seed=s, n=meta["n"], d=meta["d"], m_cold=int(rep_c.m_final), m0=int(m0), pred=float(pred),
                        m_warm=int(rep_w.m_final), cold_ms=1e3 * t_c, warm_ms=1e3 * t_w,
                        cold_passes=int(rep_c.grad_passes), warm_passes=int(rep_w.grad_passes),
                        cold_levels=int(rep_c.n_levels), warm_levels=int(rep_w.n_levels),
                        warm_status=int(rep_w.status)))
        del A, b
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=512)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args(argv)

    from . import ihs

    ctx = ihs.Context(kind="srht", variant="gd")
    tr_seeds = list(range(1000, 1000 + args.train))
    ho_seeds = list(range(900000, 900000 + args.heldout))
    t0 = time.time()
    Xtr, ytr, rows_tr, _ = build_set(ctx, tr_seeds)
    Xho, yho, rows_ho, ho_seeds = build_set(ctx, ho_seeds)
    t_data = time.time() - t0
    params, hist = train(ctx, Xtr, ytr, args.steps, args.lr, args.batch, args.seed)
    pred_tr = predict(ctx, params, Xtr)
    pred_ho = predict(ctx, params, Xho)
    cmp = compare_heldout(ctx, params, ho_seeds, rows_ho)
    summary = dict(
        train_mse=float(np.mean((pred_tr - ytr) ** 2)),
        heldout_mse=float(np.mean((pred_ho - yho) ** 2)),
        heldout_mse_constant=float(np.mean((np.mean(ytr) - yho) ** 2)),
        heldout_cold_ms=float(sum(c["cold_ms"] for c in cmp)),
        heldout_warm_ms=float(sum(c["warm_ms"] for c in cmp)),
        heldout_cold_passes=int(sum(c["cold_passes"] for c in cmp)),
        heldout_warm_passes=int(sum(c["warm_passes"] for c in cmp)),
        heldout_overshoot=int(sum(1 for c in cmp if c["m_warm"] > c["m_cold"])),
        heldout_faster=int(sum(1 for c in cmp if c["warm_ms"] < c["cold_ms"])),
        heldout_count=len(cmp),
        data_seconds=t_data,
    )
    doc = dict(network="11-64-64-1 tanh", features="log n, log d, log nu, log sigma_k of a 32-row Gaussian probe, "
                                                   "k = 1 2 3 4 6 8 12 16",
               label="log2 m_final of a cold SRHT gradient-IHS solve", sketch="srht", variant="gd",
               tol=float(ctx.params.tol), train_seeds=[tr_seeds[0], tr_seeds[-1]],
               n_train=int(len(ytr)), n_heldout=int(len(yho)),
               heldout_seeds=[ho_seeds[0], ho_seeds[-1]], steps=args.steps, lr=args.lr, batch=args.batch,
               seed=args.seed, loss_history=hist, summary=summary, heldout_first64=cmp[:64],
               params=[float(v) for v in params.cpu().numpy()])
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=0)
    print(json.dumps(summary))
    ctx.destroy()


if __name__ == "__main__":
    main()
