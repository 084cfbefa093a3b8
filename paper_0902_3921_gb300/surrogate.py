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
          channels=32, layers=6, seed0=0, log=None, reservoir=0, batch=0, updates=1, lr_final=None,
          pushforward=0.0, pushforward_from=1, init=None, t_start_hi=None):
    """Trains a network on pairs (x_t, x_{t+window}) that the plain scheme
    produces.  reservoir = 0: every window's pairs of the current lattices are
    one training batch.  reservoir > 0: the pairs stream into a device
    reservoir of that many pairs (uniform reservoir sampling over every pair
    seen), and each window is followed by `updates` steps on `batch` pairs
    drawn from it without replacement, so a batch mixes times and trajectories.
    lr decays from lr to lr_final (cosine) over the run when lr_final is set.
    pushforward > 0 (reservoir only, from generation pushforward_from on):
    that fraction of the windows also adds the pair (Net(x_{t-window}),
    x_{t+window}), whose input is the network's own prediction of x_t, so the
    network learns to correct the errors it makes when applied repeatedly.
    init: an .npz written by --save to start from (its normalisation is kept).
    t_start_hi: each generation starts at a time drawn uniformly from
    [t_start, t_start_hi] (a multiple of the window), so later stages of the
    coarsening enter the data."""
    import torch
    stream = torch.cuda.Stream()
    net = lbm.Net(channels, layers, seed=seed0 + 12345)
    if init is not None:
        z = np.load(init)
        net.set_params(z["params"])
        nrm = z["normalisation"]
        net.set_normalisation(nrm[0], nrm[1], nrm[2])
    x0 = torch.empty((lattices, side, side, 4), dtype=torch.float32, device="cuda")
    x1 = torch.empty_like(x0)
    if reservoir:
        batch = batch or lattices
        buf0 = torch.empty((reservoir, side, side, 4), dtype=torch.float32, device="cuda")
        buf1 = torch.empty_like(buf0)
        xb0 = torch.empty((batch, side, side, 4), dtype=torch.float32, device="cuda")
        xb1 = torch.empty_like(xb0)
        xprev = torch.empty_like(x0)
        xhat = torch.empty_like(x0)
    rng = np.random.default_rng(seed0)
    seen = 0
    total = generations * iters * (updates if reservoir else 1)
    step = 0
    history = []
    t0 = time.time()

    def rate():
        if lr_final is None:
            return lr
        return lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * step / max(total - 1, 1)))

    for gen in range(generations):
        ts = t_start
        if t_start_hi is not None:
            ts = int(rng.integers(t_start // window, t_start_hi // window + 1)) * window
        lats = []
        for k in range(lattices):
            lat = lbm.Lattice(_params(side), stream=stream.cuda_stream)
            n, u = I.rest(2, side, side)
            lat.init_fields(n, I.spinodal(2, side, side, seed=seed0 + gen * lattices + k), u)
            lat.step(ts)
            lats.append(lat)
        for it in range(iters):
            for k, lat in enumerate(lats):
                lbm.lbm_surrogate_state(lat.handle, x0[k].data_ptr())
                lat.step(window)
                lbm.lbm_surrogate_state(lat.handle, x1[k].data_ptr())
            if gen == 0 and it == 0 and init is None:
                stream.synchronize()
                a = x0.cpu().numpy().reshape(-1, 4)
                d = (x1 - x0).cpu().numpy().reshape(-1, 4)
                net.set_normalisation(a.mean(0), a.std(0) + 1e-12, d.std(0) + 1e-12)
            if not reservoir:
                loss = net.train_step(x0.data_ptr(), x1.data_ptr(), lattices, side, side, rate(),
                                      stream=stream.cuda_stream)
                step += 1
            else:
                with torch.cuda.stream(stream):
                    def offer(a, b):
                        nonlocal seen
                        slot = seen if seen < reservoir else int(rng.integers(0, seen + 1))
                        if slot < reservoir:
                            buf0[slot].copy_(a)
                            buf1[slot].copy_(b)
                        seen += 1
                    if pushforward > 0 and gen >= pushforward_from and it > 0 and rng.random() < pushforward:
                        net.forward(xprev.data_ptr(), lattices, side, side, xhat.data_ptr(),
                                    stream=stream.cuda_stream)
                        for k in range(lattices):
                            offer(xhat[k], x1[k])
                    for k in range(lattices):
                        offer(x0[k], x1[k])
                    xprev.copy_(x0)
                    for _ in range(updates):
                        fill = min(seen, reservoir)
                        idx = rng.choice(fill, size=min(batch, fill), replace=False)
                        for b, j in enumerate(idx):
                            xb0[b].copy_(buf0[int(j)])
                            xb1[b].copy_(buf1[int(j)])
                        loss = net.train_step(xb0.data_ptr(), xb1.data_ptr(), len(idx), side, side,
                                              rate(), stream=stream.cuda_stream)
                        step += 1
            history.append(loss)
            if log and (it % 20 == 0 or it == iters - 1):
                log(f"gen {gen} iter {it} t={lats[0].t} loss {loss:.4e} lr {rate():.2e}")
        for lat in lats:
            lat.close()
    return net, {"loss_first": history[0], "loss_last": history[-1],
                 "loss_last10": float(np.mean(history[-10:])), "pairs": lattices * iters * generations,
                 "trajectories": lattices * generations, "updates": step,
                 "reservoir": reservoir, "seconds": time.time() - t0}


def evaluate(net, side=2048, seed=1000, t_start=2000, checkpoints=(4000, 8000, 16000),
             window=50, mass_tol=2e-3, phi_clamp=0.0, relax=0, log=None, late_net=None, late_from=None,
             control=False, conserve_mass=True):
    """late_net (optional) replaces net for the windows from t = late_from on.
    conserve_mass: accepted predictions are shifted to keep the sum of phi
    (off: the prediction's own change of the sum is kept, as the plain
    scheme's printed advection form does not conserve it exactly).
    control: a third lattice, the plain scheme re-initialised from its own n,
    phi, u* at t_start (populations rebuilt at equilibrium, the reconstruction
    every accepted surrogate window makes) and then advanced by the plain
    scheme: how far two plain trajectories one such perturbation apart drift,
    the floor under which no surrogate error can be judged."""
    import torch
    stream = torch.cuda.Stream()
    n, u = I.rest(2, side, side)
    phi0 = I.spinodal(2, side, side, seed=seed)
    plain = lbm.Lattice(_params(side), stream=stream.cuda_stream).init_fields(n, phi0, u)
    surr = lbm.Lattice(_params(side), stream=stream.cuda_stream).init_fields(n, phi0, u)
    plain.step(t_start)
    surr.step(t_start)
    ctrl = None
    if control:
        cn, cphi, cu = plain.moments()
        ctrl = lbm.Lattice(_params(side), stream=stream.cuda_stream).init_fields(cn, cphi, cu)
        del cn, cphi, cu
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
        if ctrl is not None:
            ctrl.step(dt)
        use = late_net if (late_net is not None and late_from is not None and t >= late_from) else net
        with torch.cuda.stream(stream):
            ev[2].record(stream)
            nwin = dt // (window + relax)
            fb = lbm.lbm_surrogate_advance(surr.handle, use, nwin, window, mass_tol, conserve_mass,
                                           phi_clamp, relax_steps=relax)
            if dt - nwin * (window + relax):
                surr.step(dt - nwin * (window + relax))
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
               "sum_phi_start": float(phi0.sum()), "fallbacks": fb, "windows": dt // (window + relax),
               "ms_plain": tp, "ms_surrogate": ts}
        if ctrl is not None:
            _, pc, _ = ctrl.moments()
            _, Sc = OB.structure_factor(pc)
            row["L_control"] = OB.domain_size(pc)
            row["S_rel_l2_control"] = float(np.linalg.norm(Sc - Sp) / np.linalg.norm(Sp))
        rows.append(row)
        if log:
            log(json.dumps(row))
        t = tc
    plain.close()
    surr.close()
    if ctrl is not None:
        ctrl.close()
    return {"side": side, "checkpoints": rows, "speedup": tp_total / ts_total,
            "fallbacks": fb_total, "ms_plain": tp_total, "ms_surrogate": ts_total}


def load_net(path, channels=32, layers=6):
    """A network with the parameters and normalisation written by --save."""
    z = np.load(path)
    net = lbm.Net(channels, layers, seed=0)
    net.set_params(z["params"])
    nrm = z["normalisation"]
    net.set_normalisation(nrm[0], nrm[1], nrm[2])
    return net


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
    ap.add_argument("--relax", type=int, default=0, help="plain LB steps after each prediction, before the check")
    ap.add_argument("--reservoir", type=int, default=0, help="pairs kept for sampling (0: none)")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--updates", type=int, default=1, help="training steps per window")
    ap.add_argument("--lr-final", type=float, default=None)
    ap.add_argument("--pushforward", type=float, default=0.0,
                    help="fraction of windows that add (Net(x_{t-w}), x_{t+w}) pairs")
    ap.add_argument("--pushforward-from", type=int, default=1, help="first generation with them")
    ap.add_argument("--save", default=None, help="write the trained parameters (.npz)")
    ap.add_argument("--init", default=None, help="start training from these parameters (.npz)")
    ap.add_argument("--t-start", type=int, default=2000, help="LB step of the first training window")
    ap.add_argument("--t-start-hi", type=int, default=None,
                    help="draw each generation's first window uniformly from [t-start, t-start-hi]")
    ap.add_argument("--seed0", type=int, default=0, help="first training seed")
    ap.add_argument("--late", default=None, help="parameters (.npz) used from --late-from on")
    ap.add_argument("--late-from", type=int, default=16000)
    ap.add_argument("--control", action="store_true",
                    help="also run the plain scheme re-initialised from its own moments at the start")
    ap.add_argument("--load", default=None, help="evaluate parameters written by --save")
    ap.add_argument("--no-conserve-mass", action="store_true",
                    help="keep the prediction's own change of the sum of phi")
    args = ap.parse_args()
    if args.load:
        net = load_net(args.load)
        hist = {"loaded": args.load}
    else:
        net, hist = train(args.side, args.lattices, args.generations, args.iters, window=args.window,
                          lr=args.lr, log=lambda m: print(m, flush=True), reservoir=args.reservoir,
                          batch=args.batch, updates=args.updates, lr_final=args.lr_final,
                          pushforward=args.pushforward, pushforward_from=args.pushforward_from,
                          init=args.init, t_start=args.t_start, t_start_hi=args.t_start_hi,
                          seed0=args.seed0)
    if args.save:
        np.savez(args.save, params=net.get_params(), normalisation=np.asarray(net.normalisation()))
    late = None
    if args.late:
        late = load_net(args.late)
    res = evaluate(net, args.eval_side, checkpoints=tuple(int(c) for c in args.checkpoints.split(",")),
                   window=args.window, mass_tol=args.mass_tol, phi_clamp=args.phi_clamp,
                   relax=args.relax, log=lambda m: print(m, flush=True), late_net=late,
                   late_from=args.late_from if late is not None else None, control=args.control,
                   conserve_mass=not args.no_conserve_mass)
    print(json.dumps({"training": hist, "evaluation": res, "window": args.window, "relax": args.relax}),
          flush=True)


if __name__ == "__main__":
    main()
