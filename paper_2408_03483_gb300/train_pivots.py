"""Train the learned-pivot network on the converged pivot sets of plain crosses.

Data: plain solvers (nonlinear SWE, WENO5 by maxvol cross) on seeded bump
instances shaped like the 256^2 workload record, for every cross, the index
features of its initial TT and which indices ended in its converged column
pivot set (tt_fv_record_pivots).  Training: minibatch Adam on the GPU through
tt_mlp_grad / tt_mlp_adam.  The parameters are written to an .npz file that
PivotNet(params=...) loads.

    python -m paper_2408_03483_gb300.train_pivots --out pivot_net.npz
"""
import argparse
import time

import numpy as np


def instance(n, seed, cap=32):
    from synth import initial_tt
    w = dict(eqn="nonlinear", scheme="weno5", n=n, steps=1, tol=1e-8, cap=cap, ic="bumps", amp=0.1,
             amp_range=(0.01, 0.1), nbumps=1 + seed % 3, seed=seed, cfl=0.4, f=0.0)
    Q, p = initial_tt(w)
    return w, Q, p


def solver(api, w, Q, p, pivots="maxvol"):
    q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
    return api.Solver(q0, "nonlinear", "weno5", w["n"], p["dt"], w["tol"], w["cap"], g=p["g"], H=p["H"], f=p["f"],
                      seed=0, pivots=pivots)


def generate(api, sizes=(128, 256), seeds=range(20000, 20008), steps=3):
    """Rows (features, labels) recorded from plain solver runs."""
    Xs, ys = [], []
    for n in sizes:
        for sd in seeds:
            w, Q, p = instance(n, sd)
            s = solver(api, w, Q, p)
            s.record_pivots(True)
            s.step(steps)
            X, y = s.take_pivots()
            s.close()
            Xs.append(X)
            ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def _init_params(seed):
    # He-uniform weights, zero biases (the same recipe the tests' oracle uses)
    rng = np.random.default_rng(seed)

    def u(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape).astype(np.float32)

    return dict(W1=u(14, (14, 256)), b1=np.zeros(256, np.float32), W2=u(256, (256, 256)),
                b2=np.zeros(256, np.float32), w3=u(256, (256,)), b3=np.zeros(1, np.float32))


def fit(api, X, y, epochs=8, batch=8192, lr=2e-3, seed=0):
    """Minibatch Adam over the rows on the GPU; returns (params, losses)."""
    import torch
    net = api.PivotNet(_init_params(seed))
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    rng = np.random.default_rng(seed + 1)
    losses = []
    m = X.shape[0]
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(m)).cuda()
        tot = 0.0
        nb = 0
        for b0 in range(0, m, batch):
            idx = perm[b0:b0 + batch]
            loss = net.train_step(Xd[idx].contiguous(), yd[idx].contiguous(), lr)
            tot += float(loss.cpu()[0])
            nb += 1
        losses.append(tot / max(nb, 1))
    return net.host(), losses


def evaluate(api, params, sizes=(256,), seeds=range(30000, 30004), steps=3):
    """Plain vs learned start on held-out instances: cross sweeps per call,
    accepted proposals, wall time, and the two runs' relative difference."""
    import torch
    out = []
    net = api.PivotNet(params)
    for n in sizes:
        for sd in seeds:
            w, Q, p = instance(n, sd)
            res = {}
            for mode in ("maxvol", "learned"):
                s = solver(api, w, Q, p, pivots=mode)
                if mode == "learned":
                    s.set_pivot_net(net)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.step(steps)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                st = s.stats()
                res[mode] = dict(sec=dt, sweeps=st["cross_sweeps"], calls=st["cross_calls"],
                                 learned=st["learned_calls"], accepted=st["learned_accepted"],
                                 state=[q.full().numpy() for q in s.get()])
                s.close()
            scale = np.linalg.norm(res["maxvol"]["state"][0])
            diff = max(np.linalg.norm(a - b) for a, b in zip(res["maxvol"]["state"], res["learned"]["state"])) / scale
            out.append(dict(n=n, seed=sd, diff=float(diff),
                            **{f"{k}_{m}": v for m in res for k, v in res[m].items() if k != "state"}))
    return out


def main():
    from . import api
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="pivot_net.npz")
    ap.add_argument("--sizes", default="128,256")
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=8)
    args = ap.parse_args()
    sizes = tuple(int(v) for v in args.sizes.split(","))
    t0 = time.perf_counter()
    X, y = generate(api, sizes, range(20000, 20000 + args.seeds), args.steps)
    t1 = time.perf_counter()
    params, losses = fit(api, X, y, epochs=args.epochs)
    t2 = time.perf_counter()
    np.savez(args.out, **params)
    ev = evaluate(api, params)
    print(dict(rows=int(X.shape[0]), positives=int(y.sum()), gen_s=round(t1 - t0, 2), train_s=round(t2 - t1, 2),
               losses=[round(v, 5) for v in losses]))
    for e in ev:
        print(e)


if __name__ == "__main__":
    main()
