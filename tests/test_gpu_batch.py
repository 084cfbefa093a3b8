"""GPU parity of the batched engine (independent lattices of uneven size
advanced together: the persistent kernel, or the tiled path of TMA-staged and
tile-kernel collides and wavefront FD launches) against the FP64 oracle,
instance by instance."""
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


def _instance_fields(Lx, Ly, R, seed):
    op = O.Params(Lx=Lx, Ly=Ly, **CFG1)
    phi = I.drop(2, Lx, Ly, R=R, phi0=O.phi0_of(op), xi=O.xi_of(op))
    phi = phi + 0.01 * (I.uniform01(seed, Lx * Ly).reshape(Ly, Lx) - 0.5)
    n, u = I.rest(2, Lx, Ly)
    return n, phi, u


def _oracle_run(Lx, Ly, g, fs, fields, steps, m=4):
    op = O.Params(Lx=Lx, Ly=Ly, m=m, g=(g[0], g[1], 0.0), force_steps=fs, **CFG1)
    st = O.State.create(op, *fields)
    st.run(steps)
    n, u = st.moments()
    return n, st.phi, u


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_fp64_matches_oracle(graphs):
    insts = [(37, 23, (2e-5, 0.0), 12), (3, 3, (0.0, 0.0), 0), (64, 48, (0.0, 1e-5), 40),
             (5, 70, (0.0, 0.0), 0), (96, 33, (1e-5, -1e-5), 7), (32, 32, (0.0, 0.0), 0),
             (130, 17, (3e-5, 0.0), 100)]
    common = lbm.LbmParams(precision=lbm.LBM_F64, fd_substeps=4, **CFG1)
    b = lbm.Batch(common, insts)
    b.set_graphs(graphs)
    fields = []
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        f = _instance_fields(Lx, Ly, R=min(Lx, Ly) / 4, seed=k)
        fields.append(f)
        b.init_fields(k, *f)
    b.step(9).step(21)  # the force of some instances switches off inside a call
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        rn, rphi, ru = _oracle_run(Lx, Ly, g, fs, fields[k], 30)
        gn, gphi, gu = b.moments(k)
        assert np.max(np.abs(gphi - rphi)) <= 1e-11, k
        assert np.max(np.abs(gu - ru)) <= 1e-12, k
        assert np.max(np.abs(gn - rn)) <= 1e-11, k
    b.close()


def test_batch_flux_variant_odd_substeps_fp64():
    """The conservative advection form and m = 5 (sweeps of 2 + 2 + 1 FD
    substeps over the shared-memory tiles), on instances smaller than the
    halo (4 x 3), one tile (50 x 20) and several tiles (150 x 70)."""
    insts = [(4, 3, (0.0, 0.0), 0), (50, 20, (1e-5, 0.0), 6), (150, 70, (0.0, -2e-5), 100)]
    common = lbm.LbmParams(precision=lbm.LBM_F64, fd_substeps=5, adv_variant=1, **CFG1)
    b = lbm.Batch(common, insts)
    fields = []
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        f = _instance_fields(Lx, Ly, R=min(Lx, Ly) / 4, seed=10 + k)
        fields.append(f)
        b.init_fields(k, *f)
    b.step(13)
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        op = O.Params(Lx=Lx, Ly=Ly, m=5, adv_variant=1, g=(g[0], g[1], 0.0), force_steps=fs, **CFG1)
        st = O.State.create(op, *fields[k])
        st.run(13)
        rn, ru = st.moments()
        gn, gphi, gu = b.moments(k)
        assert np.max(np.abs(gphi - st.phi)) <= 1e-11, k
        assert np.max(np.abs(gu - ru)) <= 1e-12, k
        assert np.max(np.abs(gn - rn)) <= 1e-11, k
    b.close()


def test_batch_config_fp32_sampled_instances():
    """512 instances, sides in {32, 48, ..., 256}, drop radius in [6, side/3],
    half of them pushed by g_x = 1e-5 (here for the first 40 of 60 steps).
    Eight sampled instances are compared with the oracle at the FP32 bar."""
    desc = I.batch_instances(512, seed=0)
    insts = [(d["side"], d["side"], (1e-5 if d["forced"] else 0.0, 0.0),
              40 if d["forced"] else 0) for d in desc]
    common = lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG1)
    b = lbm.Batch(common, insts)
    sample = sorted(range(512), key=lambda k: desc[k]["side"])[:6] + [7, 300]
    fields = {}
    for k in range(512):
        d = desc[k]
        f = _instance_fields(d["side"], d["side"], d["R"], seed=k)
        if k in sample:
            fields[k] = f
        b.init_fields(k, *f)
    b.step(30).step(30)
    shape = b.shape()
    assert shape["sites"] == sum(d["side"] ** 2 for d in desc)
    for k in sample:
        Lx, Ly, g, fs = insts[k]
        rn, rphi, ru = _oracle_run(Lx, Ly, g, fs, fields[k], 60)
        gn, gphi, gu = b.moments(k)
        umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
        assert np.max(np.abs(gphi - rphi)) <= 1e-5, k
        assert np.max(np.abs(gu - ru)) <= 1e-3 * umax, k
    b.close()


TILED_INSTS = [(12, 20, (0.0, 0.0), 0), (32, 48, (1e-5, 0.0), 12), (100, 36, (0.0, -2e-5), 40),
               (116, 130, (2e-5, 1e-5), 5), (256, 80, (0.0, 0.0), 0), (48, 3, (1e-5, 0.0), 100),
               (64, 64, (0.0, 1e-5), 30)]


@pytest.mark.parametrize("graphs,tma", [(True, True), (False, True), (True, False)])
def test_tiled_batch_matches_oracle_fp32(graphs, tma, monkeypatch):
    """The tiled path against the oracle at the FP32 bar: the TMA collide
    for the instances at least 64 on a side and the tile kernel for the rest
    (or the tile kernel for all), two-substep wavefront FD launches; an
    instance narrower than one strip (12 wide: the strip wraps around it),
    ragged tiles, strips and segments, a 3-row instance, and body forces
    switching off inside a call."""
    monkeypatch.setenv("HLBM_BATCH_PATH", "tiled")
    if not tma:
        monkeypatch.setenv("HLBM_BATCH_NO_TMA", "1")
    common = lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG1)
    b = lbm.Batch(common, TILED_INSTS)
    b.set_graphs(graphs)
    assert b.shape()["threads"] == 0  # the tiled path
    fields = []
    for k, (Lx, Ly, g, fs) in enumerate(TILED_INSTS):
        f = _instance_fields(Lx, Ly, R=max(2, min(Lx, Ly) / 4), seed=30 + k)
        fields.append(f)
        b.init_fields(k, *f)
    b.step(9).step(21)
    for k, (Lx, Ly, g, fs) in enumerate(TILED_INSTS):
        rn, rphi, ru = _oracle_run(Lx, Ly, g, fs, fields[k], 30)
        gn, gphi, gu = b.moments(k)
        umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
        assert np.max(np.abs(gphi - rphi)) <= 1e-5, k
        assert np.max(np.abs(gu - ru)) <= 1e-3 * umax, k
        assert np.max(np.abs(gn - rn)) <= 1e-5, k
    b.close()


def test_tiled_batch_many_shapes_fp32(monkeypatch):
    """The TMA collide's per-shape tensor maps: 26 distinct shapes (more than
    one launch's 24 slots) and repeated shapes (instances at j > 0 of a
    shape, listed apart from one another), each instance against the oracle."""
    monkeypatch.setenv("HLBM_BATCH_PATH", "tiled")
    shapes = [(64 + 4 * (a % 7), 64 + 4 * (a // 7)) for a in range(26)]
    insts = [(Lx, Ly, (1e-5 if k % 3 == 0 else 0.0, 0.0), 4 if k % 3 == 0 else 0)
             for k, (Lx, Ly) in enumerate(shapes + [shapes[0], shapes[25], shapes[0], shapes[7]])]
    common = lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG1)
    b = lbm.Batch(common, insts)
    assert b.shape()["threads"] == 0
    fields = []
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        f = _instance_fields(Lx, Ly, R=12.0, seed=60 + k)
        fields.append(f)
        b.init_fields(k, *f)
    b.step(8)
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        rn, rphi, ru = _oracle_run(Lx, Ly, g, fs, fields[k], 8)
        gn, gphi, gu = b.moments(k)
        umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
        assert np.max(np.abs(gphi - rphi)) <= 1e-5, k
        assert np.max(np.abs(gu - ru)) <= 1e-3 * umax, k
    b.close()


@pytest.mark.parametrize("kw", [dict(fd_substeps=5), dict(adv_variant=1)])
def test_tiled_batch_falls_back_when_not_eligible(kw, monkeypatch):
    """Odd m or the flux form: the persistent kernel runs even when the tiled
    path is asked for."""
    monkeypatch.setenv("HLBM_BATCH_PATH", "tiled")
    args = dict(CFG1, precision=lbm.LBM_F32DEV, fd_substeps=4)
    args.update(kw)
    b = lbm.Batch(lbm.LbmParams(**args), [(32, 32, (0.0, 0.0), 0)])
    assert b.shape()["threads"] > 0
    b.close()


def test_persistent_path_forced_fp32(monkeypatch):
    """HLBM_BATCH_PATH=persistent keeps the persistent kernel on an eligible
    batch, which still meets the FP32 bar."""
    monkeypatch.setenv("HLBM_BATCH_PATH", "persistent")
    insts = TILED_INSTS[:4]
    b = lbm.Batch(lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG1), insts)
    assert b.shape()["threads"] > 0
    fields = []
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        f = _instance_fields(Lx, Ly, R=max(2, min(Lx, Ly) / 4), seed=90 + k)
        fields.append(f)
        b.init_fields(k, *f)
    b.step(20)
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        rn, rphi, ru = _oracle_run(Lx, Ly, g, fs, fields[k], 20)
        gn, gphi, gu = b.moments(k)
        assert np.max(np.abs(gphi - rphi)) <= 1e-5, k
    b.close()


def test_batch_equals_single_lattices_fp64():
    insts = [(48, 40, (1e-5, 0.0), 5), (33, 50, (0.0, 0.0), 0)]
    common = lbm.LbmParams(precision=lbm.LBM_F64, fd_substeps=4, **CFG1)
    b = lbm.Batch(common, insts)
    outs = []
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        f = _instance_fields(Lx, Ly, R=8, seed=10 + k)
        b.init_fields(k, *f)
        lat = lbm.Lattice(lbm.LbmParams(Lx=Lx, Ly=Ly, precision=lbm.LBM_F64, fd_substeps=4,
                                        g=(g[0], g[1], 0.0), force_steps=fs, **CFG1))
        lat.init_fields(*f).step(20)
        outs.append(lat.moments())
        lat.close()
    b.step(20)
    for k in range(2):
        for x, y in zip(b.moments(k), outs[k]):
            np.testing.assert_allclose(x, y, rtol=0, atol=1e-12)


def test_batch_rejects_bad_instances():
    common = lbm.LbmParams(precision=lbm.LBM_F32DEV, **CFG1)
    with pytest.raises(lbm.LbmError):
        lbm.Batch(common, [(2, 10, (0.0, 0.0), 0)])
    with pytest.raises(lbm.LbmError):
        lbm.Batch(lbm.LbmParams(precision=lbm.LBM_F16DEV, **CFG1), [(10, 10, (0.0, 0.0), 0)])
    b = lbm.Batch(common, [(10, 10, (0.0, 0.0), 0)])
    with pytest.raises(lbm.LbmError):
        b.step(1)  # not initialised
    b.close()
