"""Spurious-velocity studies of Sec. III on the GPU path (FP64 storage).

The equilibrated circular drop of Sec. III: diameter 64 on a 128 x 128
periodic lattice, -a = b = 1e-3, kappa = -3a, Gamma = 5, n = 1, u = 0,
phi = phi0 tanh((R - r)/xi) at t = 0 (the paper does not print its initial
profile).  The observable is |u*_max| / c_s (Table I, Fig. 4).

  table1     the printed optimal (N, Q) per tau (Table I), run to the
             equilibrium criterion below;
  fig4       SC (N, Q) = (1/2, 1) against OC (Table I's pair) at the six
             tau of Table I, with the FD operators as printed (stencil_fd 0)
             and with the stencil operators in Eqs. 33 and 36 (stencil_fd 1);
  nq_scan    |u*_max| / c_s over an (N, Q) grid at tau = 1, and the pair
             (7/12, 7/6) that the Taylor analysis of Eq. 39 gives.

Equilibrium criterion (the paper gives none): the run continues in windows
of `window` LB steps (default 10 000) until |u*_max| changes by less than
`rel_tol` (0.2 %) of itself over one window, after at least `min_steps`
(40 000), or `max_steps` (400 000) is reached; the history is returned so the
convergence can be read.

Run:  python -m paper_0902_3921_gb300.studies table1|fig4|nq_scan
Everything goes through the library's C ABI (paper_0902_3921_gb300.lbm).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from . import lbm

PAPER = dict(a=-1e-3, b=1e-3, kappa=3e-3, Gamma=5.0)
L, R_DROP = 128, 32
SC = (0.5, 1.0)
# Table I: tau -> (N, Q, |u*_max| / c_s)
TABLE1 = {0.6: (0.3, 3.0, 1.753e-4), 0.8: (0.3, 2.5, 6.03e-5), 1.0: (0.3, 2.5, 3.65e-5),
          1.2: (0.3, 2.5, 2.67e-5), 5.0: (0.3, 2.5, 8.8e-6), 10.0: (0.3, 2.0, 6.2e-6)}
CS = 1.0 / math.sqrt(3.0)


def drop_run(tau, N, Q, stencil_fd=0, window=10000, rel_tol=2e-3, max_steps=400000,
             min_steps=40000, fixed_steps=None):
    """|u*_max| / c_s of the Sec. III drop, sampled every `window` steps.
    Stops at the equilibrium criterion (relative change < rel_tol over one
    window, after min_steps) or at max_steps; fixed_steps runs exactly that
    many steps.  Returns dict(umax, steps, converged, history[(t, umax)])."""
    p = lbm.LbmParams(Lx=L, Ly=L, tau=tau, N=N, Q=Q, precision=lbm.LBM_F64, stencil_fd=stencil_fd,
                      **PAPER)
    xi = math.sqrt(-2.0 * PAPER["kappa"] / PAPER["a"])
    phi = I.drop(2, L, L, R=R_DROP, phi0=1.0, xi=xi)
    n, u = I.rest(2, L, L)
    lat = lbm.Lattice(p).init_fields(n, phi, u)
    hist, t, prev, converged = [], 0, None, False
    end = fixed_steps if fixed_steps is not None else max_steps
    while t < end:
        k = min(window, end - t)
        lat.step(k)
        t += k
        um = lat.diagnostics()["u_max"] / CS
        hist.append((t, um))
        if fixed_steps is None and prev is not None and t >= min_steps and abs(um - prev) <= rel_tol * um:
            converged = True
            break
        prev = um
    lat.close()
    return {"umax": hist[-1][1], "steps": t, "converged": converged, "history": hist}


def table1(**kw):
    rows = []
    for tau, (N, Q, paper) in TABLE1.items():
        r = drop_run(tau, N, Q, **kw)
        rows.append({"tau": tau, "N": N, "Q": Q, "paper": paper, **r, "ratio": r["umax"] / paper})
    return rows


def fig4(taus=tuple(TABLE1), steps=40000, check_tau=1.0):
    """SC and OC at each tau after `steps`: OC with the FD operators as printed
    and with stencil_fd; SC once (its stencils are the printed operators, so
    stencil_fd leaves it unchanged: checked at check_tau).  The paper's Fig. 4
    has SC about ten times OC over the whole tau range."""
    rows = []
    for tau in taus:
        N, Q, _ = TABLE1[tau]
        sc = drop_run(tau, *SC, fixed_steps=steps)
        oc0 = drop_run(tau, N, Q, stencil_fd=0, fixed_steps=steps)
        oc1 = drop_run(tau, N, Q, stencil_fd=1, fixed_steps=steps)
        row = {"tau": tau, "steps": steps, "sc": sc["umax"], "oc_printed": oc0["umax"],
               "oc_stencil_fd": oc1["umax"], "sc_over_oc_printed": sc["umax"] / oc0["umax"],
               "sc_over_oc_stencil_fd": sc["umax"] / oc1["umax"]}
        if tau == check_tau:
            row["sc_stencil_fd"] = drop_run(tau, *SC, stencil_fd=1, fixed_steps=steps)["umax"]
        rows.append(row)
    return rows


def nq_scan(Ns=(0.2, 0.3, 0.4, 0.5), Qs=(1.0, 1.5, 2.0, 2.5, 3.0, 3.5), tau=1.0, steps=40000,
            stencil_fd=0):
    """|u*_max| / c_s after `steps` at tau over the (N, Q) grid, and the
    analytic pair (7/12, 7/6) of Eq. 39."""
    grid = {}
    for N in Ns:
        for Q in Qs:
            grid[(N, Q)] = drop_run(tau, N, Q, stencil_fd=stencil_fd, fixed_steps=steps)["umax"]
    analytic = drop_run(tau, 7 / 12, 7 / 6, stencil_fd=stencil_fd, fixed_steps=steps)["umax"]
    return {"tau": tau, "steps": steps, "grid": {f"{N},{Q}": v for (N, Q), v in grid.items()},
            "analytic_7_12_7_6": analytic, "best": min(grid, key=grid.get)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("study", choices=["table1", "fig4", "nq_scan"])
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--rel-tol", type=float, default=2e-3)
    ap.add_argument("--window", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=40000, help="fig4 and nq_scan: steps per run")
    ap.add_argument("--json", help="write the rows to this file")
    a = ap.parse_args(argv)
    t0 = time.time()
    kw = dict(max_steps=a.max_steps, rel_tol=a.rel_tol, window=a.window)
    if a.study == "table1":
        out = table1(**kw)
        for r in out:
            print(f"tau {r['tau']:5.1f}  N {r['N']}  Q {r['Q']}  |u*max|/cs {r['umax']:.3e}  "
                  f"paper {r['paper']:.3e}  ratio {r['ratio']:.2f}  steps {r['steps']}"
                  f"{'' if r['converged'] else ' (not converged)'}")
    elif a.study == "fig4":
        out = fig4(steps=a.steps)
        for r in out:
            print(f"tau {r['tau']:5.1f}  SC {r['sc']:.3e}  OC printed {r['oc_printed']:.3e} "
                  f"(SC/OC {r['sc_over_oc_printed']:.3g})  OC stencil_fd {r['oc_stencil_fd']:.3e} "
                  f"(SC/OC {r['sc_over_oc_stencil_fd']:.3g})")
    else:
        out = nq_scan(steps=a.steps)
        for k, v in out["grid"].items():
            print(f"N,Q = {k}: {v:.3e}")
        print(f"(7/12, 7/6): {out['analytic_7_12_7_6']:.3e}; best of the grid: {out['best']}")
    print(f"({time.time() - t0:.0f} s)")
    if a.json:
        with open(a.json, "w") as f:
            json.dump(out, f, default=lambda o: list(o) if isinstance(o, tuple) else str(o))


if __name__ == "__main__":
    main()
