"""Error paths on the GPU, without faulting it: a bounded device wait that is
made to give up (the TMA collide's wait for its copies, bounded to 0 ns
through HLBM_DEBUG_TMA_WAIT_NS; the kernel still lets every issued copy land
before its CTA exits), and host-side injected faults (LBM_FAULT).  Each test
checks the reported code and message, and that the handle can be freed and a
new one created and run correctly afterwards."""
import numpy as np
import pytest

import oracle as O
from paper_0902_3921_gb300 import inputs as I
from paper_0902_3921_gb300 import lbm

pytestmark = pytest.mark.gpu

CFG1 = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_0902_3921_gb300 import build as B
    B.build()
    lbm.load_library()


def _fresh_run_matches_oracle(steps=6):
    """A new handle after the fault: 128 x 96 FP32 drop against the oracle."""
    op = O.Params(Lx=128, Ly=96, m=4, **CFG1)
    phi = I.drop(2, 128, 96, R=20, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 128, 96)
    ref = O.State.create(op, n, phi, u)
    ref.run(steps)
    lat = lbm.Lattice(lbm.LbmParams(Lx=128, Ly=96, fd_substeps=4, precision=lbm.LBM_F32DEV, **CFG1))
    lat.init_fields(n, phi, u).step(steps)
    _, gphi, _ = lat.moments()
    lat.close()
    assert float(np.max(np.abs(gphi - ref.phi))) <= 1e-5


@pytest.mark.parametrize("variant", [5, 7])
def test_tma_wait_that_gives_up_reports_etimeout(variant, monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", f"4,96,2,{variant},128")
    monkeypatch.setenv("HLBM_DEBUG_TMA_WAIT_NS", "0")
    lat = lbm.Lattice(lbm.LbmParams(Lx=128, Ly=96, fd_substeps=4, precision=lbm.LBM_F32DEV, **CFG1))
    n, u = I.rest(2, 128, 96)
    lat.init_fields(n, I.spinodal(2, 128, 96, seed=1), u)
    with pytest.raises(lbm.LbmError) as ei:
        lat.step(3)
        lat.moments()
    assert ei.value.code == lbm.LBM_ETIMEOUT, str(ei.value)
    assert "wait bound" in str(ei.value)
    lat.close()
    # the next handle restores the 0.5 s bound; the context is intact
    monkeypatch.delenv("HLBM_DEBUG_TMA_WAIT_NS")
    _fresh_run_matches_oracle()


def test_fd3_copy_wait_that_gives_up_reports_etimeout(monkeypatch):
    """The pipelined 3D FD substep (one kernel a substep, its u and v rows
    staged by bulk copies): a copy wait bounded to 0 ns gives up at once,
    every CTA drains the copies it issued and returns, and the handle reports
    LBM_ETIMEOUT at the next moments call."""
    monkeypatch.setenv("HLBM_FD3_FUSED_ADV", "1")
    monkeypatch.setenv("HLBM_DEBUG_TMA_WAIT_NS", "0")
    Lx, Ly, Lz = 128, 19, 21
    lat = lbm.Lattice(lbm.LbmParams(dims=3, Lx=Lx, Ly=Ly, Lz=Lz, fd_substeps=-8, precision=lbm.LBM_F32DEV,
                                    **dict(CFG1, N=1 / 6, Q=1 / 3)))
    n, u = I.rest(3, Lx, Ly, Lz)
    lat.init_fields(n, I.spinodal(3, Lx, Ly, Lz, seed=2), u)
    with pytest.raises(lbm.LbmError) as ei:
        lat.step(2)
        lat.moments()
    assert ei.value.code == lbm.LBM_ETIMEOUT, str(ei.value)
    assert "wait bound" in str(ei.value)
    lat.close()
    monkeypatch.delenv("HLBM_DEBUG_TMA_WAIT_NS")
    monkeypatch.delenv("HLBM_FD3_FUSED_ADV")
    _fresh_run_matches_oracle()


def test_injected_partial_allocation_failure(monkeypatch):
    monkeypatch.setenv("LBM_FAULT", "alloc:3")  # phi[0] after both population buffers
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice(lbm.LbmParams(Lx=128, Ly=96, precision=lbm.LBM_F32DEV, **CFG1))
    assert ei.value.code == lbm.LBM_ENOMEM and "alloc:K" in str(ei.value)
    monkeypatch.delenv("LBM_FAULT")
    _fresh_run_matches_oracle()


def test_injected_host_to_device_failure(monkeypatch):
    lat = lbm.Lattice(lbm.LbmParams(Lx=128, Ly=96, precision=lbm.LBM_F32DEV, **CFG1))
    n, u = I.rest(2, 128, 96)
    monkeypatch.setenv("LBM_FAULT", "h2d")
    with pytest.raises(lbm.LbmError) as ei:
        lat.init_fields(n, I.spinodal(2, 128, 96, seed=1), u)
    assert ei.value.code == lbm.LBM_ECUDA and "h2d" in str(ei.value)
    monkeypatch.delenv("LBM_FAULT")
    # the error is latched: the handle refuses further work until freed
    with pytest.raises(lbm.LbmError):
        lat.step(1)
    lat.close()
    _fresh_run_matches_oracle()
