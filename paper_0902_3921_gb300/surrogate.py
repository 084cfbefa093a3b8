"""Training and evaluation of the learned surrogate (the CUDA network of
csrc/surrogate.cu) on trajectories that the method itself generates.

train(): spinodal lattices (config of the drop/spinodal workloads) run to
t_start with the plain scheme, then every window of `window` LB steps gives a
pair (x_t, x_{t+window}) per lattice, on the device, and one training step on
the batch of pairs; every `iters` windows the lattices are replaced by new
seeds (generations).  evaluate(): one large lattice advanced twice from the
same state, by the plain scheme and by the surrogate (with its residual check
and fallback), compared at checkpoints by S(k), L(t) and sum phi, with GPU
time of both.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import inputs as I
from . import lbm
from . import observables as OB

CFG = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)


def _params(side):
    return lbm.LbmParams(Lx=side, Ly=side, precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG)


def train(side=512, lattices=8, generations=2, iters=200, window=50, t_start=2000, lr=1e-3,
          channels=32, layers=6, seed0=0, log=None):
    import torch
    stream = torch.cuda.Stream()
    net = lbm.Net(channels, layers, seed=seed0 + 12345)
    x0 = torch.empty((lattices, side, side, 4), dtype=torch.float32, device="cuda")
    x1 = torch.empty_like(x0)
    history = []
    t0 = time.time()
    for gen in range(generations):
        lats = []
        for k in range(lattices):
            lat = lbm.Lattice(_params(side), stream=stream.cuda_stream)
            n, u = I.rest(2, side, side)
            lat.init_fields(n, I.spinodal(2, side, side, seed=seed0 + gen * lattices + k), u)
            lat.step(t_start)
            lats.append(lat)
        for it in range(iters):
            for k, lat in enumerate(lats):
                lbm.lbm_surrogate_state(lat.handle, x0[k].data_ptr())
                lat.step(window)
                lbm.lbm_surrogate_state(lat.handle, x1[k].data_ptr())
            if gen == 0 and it == 0:
                stream.synchronize()
                a = x0.cpu().numpy().reshape(-1, 4)
                d = (x1 - x0).cpu().numpy().reshape(-1, 4)
                net.set_normalisation(a.mean(0), a.std(0) + 1e-12, d.std(0) + 1e-12)
            loss = net.train_step(x0.data_ptr(), x1.data_ptr(), lattices, side, side, lr,
                                  stream=stream.cuda_stream)
            history.append(loss)
            if log and (it % 20 == 0 or it == iters - 1):
                log(f"gen {gen} iter {it} t={lats[0].t} loss {loss:.4e}")
        for lat in lats:
            lat.close()
    return net, {"loss_first": history[0], "loss_last": history[-1],
                 "loss_last10": float(np.mean(history[-10:])), "pairs": lattices * iters * generations,
                 "trajectories": lattices * generations, "seconds": time.time() - t0}


def evaluate(net, side=2048, seed=1000, t_start=2000, checkpoints=(4000, 8000, 16000),
             window=50, mass_tol=2e-3, phi_clamp=0.0, log=None):
    import torch
    stream = torch.cuda.Stream()
    n, u = I.rest(2, side, side)
    phi0 = I.spinodal(2, side, side, seed=seed)
    plain = lbm.Lattice(_params(side), stream=stream.cuda_stream).init_fields(n, phi0, u)
    surr = lbm.Lattice(_params(side), stream=stream.cuda_stream).init_fields(n, phi0, u)
    plain.step(t_start)
    surr.step(t_start)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    rows, t = [], t_start
    tp_total = ts_total = 0.0
    fb_total = 0
    for tc in checkpoints:
        dt = tc - t
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            plain.step(dt)
            ev[1].record(stream)
        stream.synchronize()
        with torch.cuda.stream(stream):
            ev[2].record(stream)
            fb = lbm.lbm_surrogate_advance(surr.handle, net, dt // window, window, mass_tol, True,
                                           phi_clamp)
            ev[3].record(stream)
        stream.synchronize()
        tp, ts = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
        tp_total += tp
        ts_total += ts
        fb_total += fb
        _, pp, _ = plain.moments()
        _, ps, _ = surr.moments()
        kp, Sp = OB.structure_factor(pp)
        _, Ss = OB.structure_factor(ps)
        row = {"t": tc, "L_plain": OB.domain_size(pp), "L_surrogate": OB.domain_size(ps),
               "S_rel_l2": float(np.linalg.norm(Ss - Sp) / np.linalg.norm(Sp)),
               "sum_phi_plain": float(pp.sum()), "sum_phi_surrogate": float(ps.sum()),
               "sum_phi_start": float(phi0.sum()), "fallbacks": fb, "windows": dt // window,
               "ms_plain": tp, "ms_surrogate": ts}
        rows.append(row)
        if log:
            log(json.dumps(row))
        t = tc
    plain.close()
    surr.close()
    return {"side": side, "checkpoints": rows, "speedup": tp_total / ts_total,
            "fallbacks": fb_total, "ms_plain": tp_total, "ms_surrogate": ts_total}


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--lattices", type=int, default=8)
    ap.add_argument("--generations", type=int, default=2)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--eval-side", type=int, default=2048)
    ap.add_argument("--checkpoints", default="4000,8000,16000")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--window", type=int, default=50)
    ap.add_argument("--mass-tol", type=float, default=2e-3)
    ap.add_argument("--phi-clamp", type=float, default=0.0)
    args = ap.parse_args()
    net, hist = train(args.side, args.lattices, args.generations, args.iters, window=args.window,
                      lr=args.lr, log=lambda m: print(m, flush=True))
    res = evaluate(net, args.eval_side, checkpoints=tuple(int(c) for c in args.checkpoints.split(",")),
                   window=args.window, mass_tol=args.mass_tol, phi_clamp=args.phi_clamp,
                   log=lambda m: print(m, flush=True))
    print(json.dumps({"training": hist, "evaluation": res, "window": args.window}), flush=True)


if __name__ == "__main__":
    main()
