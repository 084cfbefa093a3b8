"""Sec. III spurious-velocity studies on the GPU path (FP64 storage), run
through paper_0902_3921_gb300.studies (also a command-line tool).

  * Table I: the printed optimal (N, Q) per tau, run to the equilibrium
    criterion of the studies module (|u*_max| changes by < 0.2 % over 10 000
    steps), compared with the printed values (tests/golden).
  * Fig. 4: SC against OC at the six tau, with the FD operators as printed
    and with stencil_fd (the stencil operators in Eqs. 33 and 36).
  * The (N, Q) scan at tau = 1 and the pair (7/12, 7/6) of Eq. 39.
Each test prints its table."""
import os

import numpy as np
import pytest

from paper_0902_3921_gb300 import lbm
from paper_0902_3921_gb300 import studies as St

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_0902_3921_gb300 import build as B
    B.build()
    lbm.load_library()


def _golden():
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_spurious_velocities.txt")):
        if line.strip() and not line.startswith("#"):
            tau, N, Q, u = (float(v) for v in line.split())
            rows[tau] = (N, Q, u)
    return rows




def test_golden_matches_the_studies_table():
    assert _golden() == St.TABLE1


def test_table1_at_equilibrium():
    """Every tau reaches the criterion.  For tau = 0.6 .. 5 the equilibrium
    |u*_max|/c_s lies within a factor 1.4 of Table I (measured 1.07-1.36) and
    decreases with tau as printed.  At tau = 10 it settles 37 % below the
    printed value; it falls towards that value throughout the run (4.2e-6 at
    45 000 steps, 3.9e-6 at 160 000), so the printed 6.2e-6 is consistent with
    a shorter run (the paper gives no run length).  The bound there is
    0.55 .. 1.4."""
    rows = St.table1()
    for r in rows:
        print(f"Table I: tau {r['tau']:5.1f} N {r['N']} Q {r['Q']}: |u*_max|/c_s {r['umax']:.3e} "
              f"(paper {r['paper']:.3e}, ratio {r['ratio']:.2f}) after {r['steps']} steps")
    for r in rows:
        assert r["converged"], r["tau"]
        lo = 0.55 if r["tau"] == 10.0 else 1 / 1.4
        assert lo <= r["ratio"] <= 1.4, (r["tau"], r["ratio"])
    u = [r["umax"] for r in rows]
    assert all(x > y for x, y in zip(u[:4], u[1:5]))


def test_fig4_sc_against_oc():
    """Fig. 4 shows SC about ten times OC at every tau.  Neither reading of
    the FD operators gives that:
      * printed FD (stencil_fd 0): SC's force Laplacian is Eq. 36's 5-point
        one, the drop has an exact stationary state and SC decays far below
        OC, whose mismatched stencils keep a steady circulation (Table I's
        magnitude);
      * stencil_fd 1: the FD Laplacian is the force's lap_D for any (N, Q),
        so OC gets an exact stationary state too and decays as SC does
        (below a tenth of the printed-FD value by 40 000 steps for tau <= 1.2,
        more slowly at tau = 5 and 10).
    SC evaluates the same operators in both settings (its stencils are the
    printed ones); the tile kernel that runs stencil_fd sums the Laplacian
    in another order, so the two SC runs agree to rounding, not bitwise."""
    rows = St.fig4(steps=40000)
    for r in rows:
        print(f"Fig. 4, tau {r['tau']:5.1f}: SC {r['sc']:.3e}; OC printed {r['oc_printed']:.3e} "
              f"(SC/OC {r['sc_over_oc_printed']:.3g}); OC stencil_fd {r['oc_stencil_fd']:.3e} "
              f"(SC/OC {r['sc_over_oc_stencil_fd']:.3g})")
    for r in rows:
        # the paper's Fig. 4 has SC/OC about 10; measured 0.003-0.007 for
        # tau <= 1.2, 0.06 and 0.13 at tau = 5 and 10 (40 000 steps)
        assert r["sc_over_oc_printed"] < (0.02 if r["tau"] <= 1.2 else 0.2), r["tau"]
        assert r["oc_printed"] > 0.5 * St.TABLE1[r["tau"]][2], r["tau"]
        # still decaying at high tau after 40 000 steps
        assert r["oc_stencil_fd"] < (0.1 if r["tau"] <= 1.2 else 0.5) * r["oc_printed"], r["tau"]
        if "sc_stencil_fd" in r:
            assert abs(r["sc_stencil_fd"] - r["sc"]) <= 0.1 * r["sc"] + 5e-8


def test_nq_scan_and_the_eq39_pair():
    """At tau = 1 (40 000 steps) |u*_max| grows with Q - 1 at every N and only
    weakly with N; the pair (7/12, 7/6) from the Taylor brackets of Eq. 39
    gives a smaller spurious velocity than Table I's (0.3, 2.5)."""
    out = St.nq_scan(Ns=(0.2, 0.35, 0.5), Qs=(1.5, 2.5, 3.5), steps=40000)
    g = {tuple(float(x) for x in k.split(",")): v for k, v in out["grid"].items()}
    for (N, Q), v in sorted(g.items()):
        print(f"(N, Q) scan, tau 1: N {N} Q {Q}: |u*_max|/c_s {v:.3e}")
    print(f"(7/12, 7/6): {out['analytic_7_12_7_6']:.3e}")
    for N in (0.2, 0.35, 0.5):
        assert g[(N, 1.5)] < g[(N, 2.5)] < g[(N, 3.5)], N
    for Q in (1.5, 2.5, 3.5):
        vals = [g[(N, Q)] for N in (0.2, 0.35, 0.5)]
        assert max(vals) < 1.5 * min(vals), Q
    table_pair = St.drop_run(1.0, 0.3, 2.5, fixed_steps=40000)["umax"]
    assert out["analytic_7_12_7_6"] < 0.5 * table_pair
