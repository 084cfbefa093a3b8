"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances (written here, derived in the design notes):
  * FP64 mode: |d phi|, |d f| <= 1e-11 and |d u*| <= 1e-12 (FMA contraction and
    summation order are the only differences from the oracle);
  * FP32-deviation mode, drop configuration (64^2, R = 16, 2000 steps):
    |d phi|_inf <= 1e-5 and |d u*|_inf <= 1e-3 max|u*_oracle|;
  * FP16-deviation mode: error reported, bounded loosely.
"""
import os

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


def _pair(Lx, Ly, Lz=1, dims=2, m=4, precision=lbm.LBM_F64, **kw):
    """Matching oracle / library parameters."""
    op = O.Params(dims=dims, Lx=Lx, Ly=Ly, Lz=Lz if dims == 3 else 1, m=m, **kw)
    lp = lbm.LbmParams(dims=dims, Lx=Lx, Ly=Ly, Lz=Lz if dims == 3 else 1, fd_substeps=-m,
                       precision=precision, **kw)
    return op, lp


def _run_both(op, lp, n, phi, u, steps, chunks=None, graphs=True):
    ref = O.State.create(op, n, phi, u)
    ref.run(steps)
    lat = lbm.Lattice(lp)
    lbm.lbm_set_graphs(lat.handle, graphs)
    lat.init_fields(n, phi, u)
    for c in (chunks or [steps]):
        lat.step(c)
    return ref, lat


def _errors(ref, lat):
    rn, ru = ref.moments()
    gn, gphi, gu = lat.moments()
    return (float(np.max(np.abs(gphi - ref.phi))), float(np.max(np.abs(gu - ru))),
            float(np.max(np.abs(gn - rn))))


@pytest.fixture(scope="module")
def drop_2000():
    """The FP64 drop configuration: 64^2, R = 16, 2000 steps, oracle side."""
    op = O.Params(Lx=64, Ly=64, m=4, **CFG1)
    phi = I.drop(2, 64, 64, R=16, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 64, 64)
    ref = O.State.create(op, n, phi, u)
    ref.run(2000)
    return op, (n, phi, u), ref


def test_drop_config_fp64(drop_2000):
    op, (n, phi, u), ref = drop_2000
    lat = lbm.Lattice(lbm.LbmParams(Lx=64, Ly=64, fd_substeps=4, precision=lbm.LBM_F64, **CFG1))
    lat.init_fields(n, phi, u).step(2000)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (dphi, du, dn)
    f = lat.populations()
    assert np.max(np.abs(f - ref.f)) <= 1e-11
    # FP64 diagnostics against the oracle's
    dg = lat.diagnostics()
    do = O.diagnostics(op, ref.f, ref.phi, ref.t, np.array([32.0, 32.0, 0.0]))
    for k in ("sum_n", "sum_phi", "u_max", "dp", "area", "R_eff"):
        assert dg[k] == pytest.approx(do[k], rel=1e-10, abs=1e-12), k
    np.testing.assert_allclose(dg["r_cm"], do["r_cm"], atol=1e-9)
    np.testing.assert_allclose(dg["v_f"], do["v_f"], atol=1e-12)
    np.testing.assert_allclose(dg["momentum"], do["momentum"], atol=1e-12)
    assert dg["nonfinite"] == 0


def test_drop_config_fp32_deviation(drop_2000):
    """The stated bar: after 2000 steps |d phi|_inf <= 1e-5 and
    |d u*|_inf <= 1e-3 max |u*_oracle|."""
    op, (n, phi, u), ref = drop_2000
    _, ru = ref.moments()
    lat = lbm.Lattice(lbm.LbmParams(Lx=64, Ly=64, fd_substeps=4, precision=lbm.LBM_F32DEV,
                                    **CFG1))
    lat.init_fields(n, phi, u).step(2000)
    dphi, du, dn = _errors(ref, lat)
    umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
    print(f"fp32dev drop 2000: |dphi|={dphi:.3e} |du|={du:.3e} umax={umax:.3e} |dn|={dn:.3e}")
    assert dphi <= 1e-5, dphi
    assert du <= 1e-3 * umax, (du, umax)


def test_drop_config_fp16_deviation(drop_2000):
    """FP16 deviations (scale 2^10): the error is stated, bounded loosely."""
    op, (n, phi, u), ref = drop_2000
    _, ru = ref.moments()
    lat = lbm.Lattice(lbm.LbmParams(Lx=64, Ly=64, fd_substeps=4, precision=lbm.LBM_F16DEV,
                                    **CFG1))
    lat.init_fields(n, phi, u).step(2000)
    dphi, du, dn = _errors(ref, lat)
    umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
    print(f"fp16dev drop 2000: |dphi|={dphi:.3e} |du|={du:.3e} umax={umax:.3e} |dn|={dn:.3e}")
    assert dphi <= 1e-2 and du <= 0.1 * umax


@pytest.mark.parametrize("Lx,Ly", [(37, 23), (3, 3), (5, 70), (96, 33), (130, 17)])
def test_ragged_sizes_fp64(Lx, Ly):
    """Sizes that are not multiples of any tile, down to 3 x 3."""
    op, lp = _pair(Lx, Ly, **CFG1)
    rng = np.random.default_rng(Lx * 100 + Ly)
    phi = 0.8 * (rng.random((Ly, Lx)) - 0.5)
    n = 1 + 0.01 * (rng.random((Ly, Lx)) - 0.5)
    u = 0.01 * (rng.random((2, Ly, Lx)) - 0.5)
    ref, lat = _run_both(op, lp, n, phi, u, 30)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (dphi, du, dn)
    assert np.max(np.abs(lat.populations() - ref.f)) <= 1e-11


@pytest.mark.parametrize("variant", ["flux", "cubic_half", "T", "force", "m1", "m5", "SC",
                                     "tau", "m9"])
def test_variants_fp64(variant):
    kw = dict(CFG1)
    m = 4
    steps, chunks = 40, None
    if variant == "flux":
        kw["adv_variant"] = 1
    elif variant == "cubic_half":
        kw["cubic_at_half"] = 1
    elif variant == "T":
        kw["T"] = 0.28
    elif variant == "force":
        kw["g"] = (2e-5, -1e-5, 0.0)
        kw["force_steps"] = 25
        chunks = [7, 30, 3]  # the force switches off inside a call
    elif variant == "m1":
        kw.update(a=-1e-3, b=1e-3, kappa=3e-3, Gamma=5.0)
        m = 1
    elif variant == "m5":
        m = 5  # two FD launches (4 + 1 substeps) per step
    elif variant == "m9":
        m = 9  # three FD launches (4 + 4 + 1)
    elif variant == "SC":
        kw.update(N=0.5, Q=1.0)
    elif variant == "tau":
        kw["tau"] = 0.7
    op, lp = _pair(48, 40, m=m, **kw)
    phi = I.drop(2, 48, 40, R=10, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 48, 40)
    u = u + 0.002 * np.sin(np.arange(48) / 5.0)[None, None, :]
    ref, lat = _run_both(op, lp, n, phi, u, steps, chunks=chunks)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (variant, dphi, du, dn)


def test_graphs_match_eager_bitwise():
    op, lp = _pair(64, 48, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.spinodal(2, 64, 48, seed=3)
    n, u = I.rest(2, 64, 48)
    outs = []
    for graphs in (True, False):
        lat = lbm.Lattice(lp)
        lbm.lbm_set_graphs(lat.handle, graphs)
        lat.init_fields(n, phi, u)
        for c in (1, 64, 65, 3, 130):
            lat.step(c)
        outs.append(lat.moments())
        lat.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_translation_equivariance_bitwise():
    op, lp = _pair(64, 48, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.spinodal(2, 64, 48, seed=5)
    n, u = I.rest(2, 64, 48)
    res = []
    for shift in ((0, 0), (7, 13)):
        lat = lbm.Lattice(lp)
        lat.init_fields(n, np.roll(phi, shift, axis=(0, 1)), u).step(100)
        res.append(lat.moments())
        lat.close()
    for a, b in zip(res[0], res[1]):
        axes = (0, 1) if a.ndim == 2 else (1, 2)
        assert np.array_equal(np.roll(a, (7, 13), axis=axes), b)


@pytest.mark.parametrize("precision", [lbm.LBM_F64, lbm.LBM_F32DEV])
def test_rest_state_gpu(precision):
    op, lp = _pair(40, 24, precision=precision, **CFG1)
    n, u = I.rest(2, 40, 24)
    phi = np.ones((24, 40))
    lat = lbm.Lattice(lp)
    lat.init_fields(n, phi, u).step(50)
    gn, gphi, gu = lat.moments()
    assert np.array_equal(gphi, phi)
    assert np.max(np.abs(gu)) < 1e-15
    assert np.max(np.abs(gn - 1)) < 1e-12


def test_spinodal_full_size_fp32():
    """The 1024 x 1024 spinodal workload in the benchmark's launch
    configuration: 5 steps against the oracle at every site."""
    op, lp = _pair(1024, 1024, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.spinodal(2, 1024, 1024, seed=0)
    n, u = I.rest(2, 1024, 1024)
    ref, lat = _run_both(op, lp, n, phi, u, 5)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-6 and du <= 1e-8 and dn <= 1e-6, (dphi, du, dn)


def test_sum_n_conserved_fp32_long():
    """Mass conservation over 2000 steps of the spinodal workload (any size)."""
    op, lp = _pair(256, 256, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.spinodal(2, 256, 256, seed=1)
    n, u = I.rest(2, 256, 256)
    lat = lbm.Lattice(lp)
    lat.init_fields(n, phi, u)
    d0 = lat.diagnostics()
    lat.step(2000)
    d1 = lat.diagnostics()
    assert abs(d1["sum_n"] - d0["sum_n"]) < 1e-6 * 65536
    assert d1["nonfinite"] == 0


def test_flux_variant_conserves_phi_fp64():
    op, lp = _pair(64, 64, adv_variant=1, **CFG1)
    phi = I.spinodal(2, 64, 64, seed=2, amp=0.1)
    n, u = I.rest(2, 64, 64)
    lat = lbm.Lattice(lp)
    lat.init_fields(n, phi, u)
    s0 = lat.diagnostics()["sum_phi"]
    lat.step(300)
    s1 = lat.diagnostics()["sum_phi"]
    assert abs(s1 - s0) < 1e-10


# ---- 3D (D3Q19) ------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(12, 10, 8), (5, 3, 7)])
def test_3d_fp64_parity(shape):
    Lx, Ly, Lz = shape
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    op, lp = _pair(Lx, Ly, Lz, dims=3, m=8, **kw)
    rng = np.random.default_rng(11)
    phi = 0.8 * (rng.random((Lz, Ly, Lx)) - 0.5)
    n = 1 + 0.01 * (rng.random((Lz, Ly, Lx)) - 0.5)
    u = 0.01 * (rng.random((3, Lz, Ly, Lx)) - 0.5)
    ref, lat = _run_both(op, lp, n, phi, u, 12)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (dphi, du, dn)
    assert np.max(np.abs(lat.populations() - ref.f)) <= 1e-11


@pytest.mark.parametrize("variant", ["T", "force", "flux"])
def test_3d_variants_fp64(variant):
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    if variant == "T":
        kw["T"] = 0.3
    elif variant == "force":
        kw.update(g=(1e-5, 2e-5, -3e-5), force_steps=4)
    else:
        kw["adv_variant"] = 1
    op, lp = _pair(20, 18, 16, dims=3, m=8, **kw)
    phi = I.drop(3, 20, 18, 16, R=5, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, 20, 18, 16)
    ref, lat = _run_both(op, lp, n, phi, u, 8)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (variant, dphi, du, dn)


@pytest.mark.parametrize("variant", ["paper", "flux"])
@pytest.mark.parametrize("fd_path,shape", [("vec", (36, 19, 21)), ("vec", (132, 10, 17)),
                                           ("scalar", (37, 18, 21)), ("tile", (37, 18, 21)),
                                           ("fused", (128, 19, 21)), ("fused", (256, 9, 13)),
                                           ("psi", (128, 19, 21)), ("psi", (256, 9, 13)),
                                           ("vec", (128, 19, 21))])
def test_3d_fp32_fd_paths(variant, fd_path, shape, monkeypatch):
    """FP32 3D against the oracle, both advection forms: the three FD passes
    with four x-sites per thread marching in z (Lx a multiple of 4; ragged in
    x against the 128-site warp, in y against 8 rows, in z against 16
    planes), the one-site-per-thread passes (any Lx), the shared-memory
    tile kernel, the advection pass followed by the fused psi / new-phi
    kernel ("psi", the default for Lx = 128 or 256), and the whole substep
    in one kernel ("fused", opt-in); both ragged in y against the rows per
    CTA (14 and 12) and in z against the planes per CTA; 9 rows: fewer than
    one CTA's."""
    if fd_path == "tile":
        monkeypatch.setenv("HLBM_FD3_TILE", "1")
    if fd_path == "fused":
        monkeypatch.setenv("HLBM_FD3_FUSED_ADV", "1")
    if fd_path == "vec" and shape[0] in (128, 256):
        monkeypatch.setenv("HLBM_FD3_UNFUSED", "1")
    Lx, Ly, Lz = shape
    kw = dict(CFG1, N=1 / 6, Q=1 / 3, adv_variant=1 if variant == "flux" else 0)
    op, lp = _pair(Lx, Ly, Lz, dims=3, m=8, precision=lbm.LBM_F32DEV, **kw)
    phi = I.drop(3, Lx, Ly, Lz, R=6, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, Lx, Ly, Lz)
    u = u + 0.002 * np.sin(np.arange(Lx) / 5.0)[None, None, None, :]
    u[1] += 0.001 * np.cos(np.arange(Lz) / 3.0)[:, None, None]
    ref, lat = _run_both(op, lp, n, phi, u, 10)
    dphi, du, dn = _errors(ref, lat)
    _, ru = ref.moments()
    umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
    assert dphi <= 1e-5 and du <= 1e-3 * umax, (variant, fd_path, dphi, du, umax)


@pytest.mark.parametrize("extra,shape", [("", (128, 19, 21)), ("", (256, 30, 17)),
                                         ("cubic_half", (256, 30, 17)), ("flux", (128, 19, 21))])
def test_3d_fused_substep_matches_two_kernel_path(extra, shape, monkeypatch):
    """The one-kernel FD substep (advection, psi and the new phi fused in
    one software-pipelined kernel; opt-in) against the advection pass
    followed by the psi / new-phi kernel: the same FP32 arithmetic per site
    (the advection of both is one device function, psi and the new phi the
    same packed operations), so after 10 LB steps the fields are equal
    bitwise; also with the cube of Eq. 36 taken from the advected phi and
    with the flux form of the advection."""
    Lx, Ly, Lz = shape
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    if extra == "cubic_half":
        kw["cubic_at_half"] = 1
    if extra == "flux":
        kw["adv_variant"] = 1
    lp = lbm.LbmParams(dims=3, Lx=Lx, Ly=Ly, Lz=Lz, fd_substeps=-8, precision=lbm.LBM_F32DEV, **kw)
    op = O.Params(dims=3, Lx=Lx, Ly=Ly, Lz=Lz, m=8, **kw)
    phi = I.drop(3, Lx, Ly, Lz, R=7, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, Lx, Ly, Lz)
    u = u + 0.003 * np.sin(np.arange(Lx) / 5.0)[None, None, None, :]
    u[2] -= 0.002 * np.cos(np.arange(Ly) / 3.0)[None, :, None]
    res = []
    for fused in (True, False):
        if fused:
            monkeypatch.setenv("HLBM_FD3_FUSED_ADV", "1")
        else:
            monkeypatch.delenv("HLBM_FD3_FUSED_ADV")
        lat = lbm.Lattice(lp)
        lat.init_fields(n, phi, u).step(10)
        res.append(lat.moments())
        lat.close()
    d = [float(np.max(np.abs(a - b))) for a, b in zip(res[0], res[1])]
    print(f"fused vs two-kernel FD, {extra or 'paper'} {shape}: |dn|={d[0]:.3e} |dphi|={d[1]:.3e} |du|={d[2]:.3e}")
    assert d == [0.0, 0.0, 0.0], d


def test_3d_drop_64_fp32_and_fp16():
    """The 64^3 copy of the 3D drop (R = 12): FP32 and FP16 deviations against
    FP64 after 20 steps; the errors are printed (stated per result)."""
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    op = O.Params(dims=3, Lx=64, Ly=64, Lz=64, m=8, **kw)
    phi = I.drop(3, 64, 64, 64, R=12, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, 64, 64, 64)
    ref = O.State.create(op, n, phi, u)
    ref.run(20)
    _, ru = ref.moments()
    umax = float(np.max(np.abs(ru)))
    for prec, bphi, bu in ((lbm.LBM_F32DEV, 1e-5, 1e-3), (lbm.LBM_F16DEV, 1e-2, 0.2)):
        lat = lbm.Lattice(lbm.LbmParams(dims=3, Lx=64, Ly=64, Lz=64, fd_substeps=8,
                                        precision=prec, **kw))
        lat.init_fields(n, phi, u).step(20)
        dphi, du, dn = _errors(ref, lat)
        print(f"3D 64^3 drop, precision {prec}: |dphi|={dphi:.3e} |du|={du:.3e} "
              f"umax={umax:.3e}")
        assert dphi <= bphi and du <= bu * umax
        lat.close()


def test_3d_drop_64_precision_over_5000_steps():
    """The 64^3 copy of the 3D drop (R = 12) over the workload's 5000 steps:
    FP32 and FP16 deviations against the FP64 path (which the short 3D
    parity tests tie to the oracle within 1e-11; the FP64 oracle itself
    would need tens of CPU minutes here).  The errors are printed (stated per
    result).  Bounds: FP32, one FP32 rounding (1e-7) of phi ~ 1 per step for
    5000 steps, |dphi| <= 5e-4, and 1 % of max|u*|; FP16 (11-bit mantissa on
    the deviations), |dphi| <= 5e-2 and 30 % of max|u*|."""
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    op = O.Params(dims=3, Lx=64, Ly=64, Lz=64, m=8, **kw)
    phi = I.drop(3, 64, 64, 64, R=12, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, 64, 64, 64)
    res = {}
    for prec in (lbm.LBM_F64, lbm.LBM_F32DEV, lbm.LBM_F16DEV):
        lat = lbm.Lattice(lbm.LbmParams(dims=3, Lx=64, Ly=64, Lz=64, fd_substeps=8,
                                        precision=prec, **kw))
        lat.init_fields(n, phi, u).step(5000)
        res[prec] = lat.moments()
        lat.close()
    rn, rphi, ru = res[lbm.LBM_F64]
    umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
    for prec, bphi, bu in ((lbm.LBM_F32DEV, 5e-4, 1e-2), (lbm.LBM_F16DEV, 5e-2, 0.3)):
        gn, gphi, gu = res[prec]
        dphi = float(np.max(np.abs(gphi - rphi)))
        du = float(np.max(np.abs(gu - ru)))
        dn = float(np.max(np.abs(gn - rn)))
        print(f"3D 64^3 drop, 5000 steps, precision {prec} vs FP64: |dphi|={dphi:.3e} "
              f"|du|={du:.3e} |dn|={dn:.3e} max|u*|={umax:.3e}")
        assert dphi <= bphi and du <= bu * umax, (prec, dphi, du, umax)


@pytest.mark.parametrize("precision", [lbm.LBM_F32DEV, lbm.LBM_F64])
def test_handle_on_torch_buffers(precision):
    """A handle that adopts torch-allocated buffers gives the same bits as one
    that owns its memory, and really works in them: after lbm_init_fields the
    torch phi plane holds phi(0)."""
    import torch
    Lx, Ly = 70, 45
    p = lbm.LbmParams(Lx=Lx, Ly=Ly, precision=precision, **CFG1)
    bp, bphi, bu = lbm.lbm_buffer_bytes(p)
    dt = torch.float64 if precision == lbm.LBM_F64 else torch.float32
    es = torch.finfo(dt).bits // 8
    bufs = {"populations": [torch.zeros(bp // es, dtype=dt, device="cuda") for _ in range(2)],
            "phi": [torch.zeros(bphi // es, dtype=dt, device="cuda") for _ in range(3)],
            "u": torch.zeros(bu // es, dtype=dt, device="cuda")}
    phi = I.drop(2, Lx, Ly, R=10, phi0=1.0, xi=1.67)
    n, u = I.rest(2, Lx, Ly)
    a = lbm.Lattice(p, buffers=bufs).init_fields(n, phi, u)
    a.synchronize()
    np.testing.assert_array_equal(bufs["phi"][0].cpu().numpy().reshape(Ly, Lx), phi.astype(
        np.float64 if precision == lbm.LBM_F64 else np.float32))
    b = lbm.Lattice(p).init_fields(n, phi, u)
    a.step(30)
    b.step(30)
    for xa, xb in zip(a.moments(), b.moments()):
        assert np.array_equal(xa, xb)
    a.close()
    b.close()
    assert torch.isfinite(bufs["populations"][0]).all()  # still usable after the handle is freed


@pytest.mark.parametrize("shape", ["1,32,4,0,32", "1,32,4,2,64", "2,32,4,4,64"])
@pytest.mark.parametrize("precision", [lbm.LBM_F64, lbm.LBM_F32DEV])
def test_stencil_fd_against_oracle(shape, precision, monkeypatch):
    """stencil_fd = 1 (the stencil operators of Eqs. 30-31 in Eqs. 33 and 36,
    Sec. II C after Eq. 36 and Sec. IV) on the tile FD kernel, against the
    oracle with the same option: FP64 at 1e-11, FP32 at the FP32 bar; a
    lattice smaller than a tile and an odd m (a remainder launch).  lap_D with
    Q = 2.5 has the largest eigenvalue 8Q = 20 (8 for the 5-point form), so
    Eq. 36 needs m = 21 here for dt x stiffness <= 1.5."""
    monkeypatch.setenv("HLBM_TUNING", shape)
    kw = dict(CFG1, stencil_fd=1)
    op, lp = _pair(70, 45, m=21, precision=precision, **kw)
    phi = I.drop(2, 70, 45, R=12, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 70, 45)
    u = u + 0.003 * np.sin(np.arange(70) / 4.0)[None, None, :]
    u[1] += 0.002 * np.cos(np.arange(45) / 3.0)[:, None]
    ref, lat = _run_both(op, lp, n, phi, u, 25)
    if precision == lbm.LBM_F64:
        dphi, du, dn = _errors(ref, lat)
        assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (shape, dphi, du, dn)
    else:
        _fp32_bar(ref, lat, shape)


def test_stencil_fd_autotuned_and_differs_from_printed():
    """An autotuned stencil_fd handle runs the tile kernel and matches the
    oracle; with OC stencils its result differs from the printed scheme's."""
    kw = dict(CFG1, stencil_fd=1)
    op, lp = _pair(96, 64, m=21, precision=lbm.LBM_F64, **kw)
    phi = I.drop(2, 96, 64, R=16, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 96, 64)
    ref, lat = _run_both(op, lp, n, phi, u, 40)
    dphi, du, _ = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12
    assert lbm.lbm_tuning(lat.handle)["fd_tile_width"] in (32, 64)
    # the automatic m follows lap_D's spectrum: stiffness 30 -> m = 20
    auto = lbm.Lattice(lbm.LbmParams(Lx=96, Ly=64, precision=lbm.LBM_F64, **kw))
    assert lbm.lbm_fd_substeps(auto.handle) == 20
    auto.close()
    op0 = O.Params(**{**op.__dict__, "stencil_fd": 0})
    ref0 = O.State.create(op0, n, phi, u)
    ref0.run(40)
    assert np.max(np.abs(ref0.phi - ref.phi)) > 1e-9


def test_checkpoint_roundtrip_bitwise(tmp_path):
    op, lp = _pair(48, 40, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.spinodal(2, 48, 40, seed=9)
    n, u = I.rest(2, 48, 40)
    a = lbm.Lattice(lp)
    a.init_fields(n, phi, u).step(100)
    path = str(tmp_path / "ck.bin")
    lbm.lbm_save(a.handle, path)
    a.step(100)
    b = lbm.Lattice(lp)
    assert lbm.lbm_load(b.handle, path) == lbm.LBM_OK
    assert b.t == 100
    b.step(100)
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    # a corrupted file is refused and leaves the handle usable
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    assert lbm.lbm_load(b.handle, path) == lbm.LBM_EINVAL
    assert "CRC mismatch" in lbm.load_library().lbm_last_error(b.handle).decode()
    b.step(1)
    assert lbm.lbm_load(b.handle, str(tmp_path / "missing.bin")) == lbm.LBM_EINVAL
    assert "cannot open" in lbm.load_library().lbm_last_error(b.handle).decode()
    b.step(1)


def test_errors_are_latched_not_fatal():
    lp = lbm.LbmParams(Lx=16, Ly=16, precision=lbm.LBM_F32DEV, **CFG1)
    lat = lbm.Lattice(lp)
    with pytest.raises(lbm.LbmError) as ei:
        lat.step(1)  # before init
    assert ei.value.code == lbm.LBM_ESTATE
    # the handle refuses further work and still frees cleanly
    with pytest.raises(lbm.LbmError):
        lat.init_fields(np.ones((16, 16)), np.zeros((16, 16)), np.zeros((2, 16, 16)))
    lat.close()


def test_nonfinite_is_reported():
    lp = lbm.LbmParams(Lx=16, Ly=16, precision=lbm.LBM_F32DEV, **CFG1)
    lat = lbm.Lattice(lp)
    phi = np.zeros((16, 16))
    phi[3, 4] = np.nan
    lat.init_fields(np.ones((16, 16)), phi, np.zeros((2, 16, 16)))
    d = lat.diagnostics()
    assert d["nonfinite"] == 1 and d["rc"] == lbm.LBM_ENONFINITE
    lat.step(1)  # still usable


# every launch shape the autotuner can pick, pinned through HLBM_TUNING
# ("FD substeps per launch, rows per warp, columns per lane, collide sites per
# thread, FD tile width")
SHAPES = ["4,16,4,2,0", "4,8,2,4,0", "2,32,4,0,0", "3,16,4,2,0", "1,64,2,1,0",
          "1,32,4,0,32", "1,32,4,2,64", "2,32,4,4,64", "4,16,2,1,0"]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [lbm.LBM_F64, lbm.LBM_F32DEV])
def test_every_launch_shape(shape, precision, monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", shape)
    kw = dict(CFG1)
    op, lp = _pair(70, 45, m=5, precision=precision, **kw)  # m = 5: a remainder launch
    phi = I.drop(2, 70, 45, R=12, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 70, 45)
    u = u + 0.003 * np.sin(np.arange(70) / 4.0)[None, None, :]
    ref, lat = _run_both(op, lp, n, phi, u, 25)
    dphi, du, dn = _errors(ref, lat)
    if precision == lbm.LBM_F64:
        assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (shape, dphi, du, dn)
    else:  # the FP32-deviation bar: |dphi| <= 1e-5, |du| <= 1e-3 max|u*|
        _, ru = ref.moments()
        umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
        assert dphi <= 1e-5 and du <= 1e-3 * umax, (shape, dphi, du, umax)
    t = lbm.lbm_tuning(lat.handle)
    assert t["fd_tile_width"] == int(shape.split(",")[4])


# FP32 block kernel shapes (substeps, region rows, warps / 8; tile 128)
BLOCK_SHAPES = ["4,80,2,1,128", "4,96,2,1,128", "4,96,4,1,128", "2,64,2,1,128", "2,80,2,1,128",
                "2,96,4,1,128", "1,64,2,1,128"]


def _fp32_bar(ref, lat, tag):
    dphi, du, dn = _errors(ref, lat)
    _, ru = ref.moments()
    umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
    assert dphi <= 1e-5 and du <= 1e-3 * umax, (tag, dphi, du, umax)


@pytest.mark.parametrize("shape", BLOCK_SHAPES)
@pytest.mark.parametrize("size", [(70, 45), (300, 217)])
def test_block_kernel_shapes(shape, size, monkeypatch):
    """The FP32 block FD kernel: a lattice smaller than one 128-column region
    (the region wraps around it) and one of several regions with ragged
    edges; m = 5 adds a remainder launch."""
    monkeypatch.setenv("HLBM_TUNING", shape)
    Lx, Ly = size
    op, lp = _pair(Lx, Ly, m=5, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.drop(2, Lx, Ly, R=min(Lx, Ly) // 4, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, Lx, Ly)
    u = u + 0.003 * np.sin(np.arange(Lx) / 4.0)[None, None, :]
    ref, lat = _run_both(op, lp, n, phi, u, 12)
    _fp32_bar(ref, lat, shape)
    assert lbm.lbm_tuning(lat.handle)["fd_tile_width"] == 128


@pytest.mark.parametrize("shape", ["4,80,2,1,128", "2,64,2,1,128", "4,96,4,1,128"])
def test_block_kernel_flux_variant(shape, monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", shape)
    op, lp = _pair(150, 90, m=4, adv_variant=1, cubic_at_half=1, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.drop(2, 150, 90, R=20, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 150, 90)
    u = u + 0.003 * np.cos(np.arange(90) / 3.0)[None, :, None]
    ref, lat = _run_both(op, lp, n, phi, u, 15)
    _fp32_bar(ref, lat, shape)


# y-marching wavefront FD kernel (tile 1): substeps per launch 4 or 2, rows =
# output rows of a segment
WAVE_SHAPES = ["4,32,4,1,1", "4,7,4,1,1", "2,16,4,1,1", "4,256,4,1,1", "2,5,4,1,1", "2,200,4,1,1"]


@pytest.mark.parametrize("shape", WAVE_SHAPES)
@pytest.mark.parametrize("size,m", [((72, 45), 5), ((300, 217), 4), ((64, 20), 6), ((412, 130), 8)])
def test_wave_kernel_shapes(shape, size, m, monkeypatch):
    """The wavefront FD kernel against the oracle: a lattice narrower than
    one strip (the strip wraps around it), strips and segments with ragged
    edges, segments taller than the lattice, and m = 5 / 6 / 8 (a remainder
    launch of 1 or 2 substeps, or two launches of 4)."""
    monkeypatch.setenv("HLBM_TUNING", shape)
    Lx, Ly = size
    op, lp = _pair(Lx, Ly, m=m, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.drop(2, Lx, Ly, R=min(Lx, Ly) // 4, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, Lx, Ly)
    u = u + 0.003 * np.sin(np.arange(Lx) / 4.0)[None, None, :]
    u[1] += 0.002 * np.cos(np.arange(Ly) / 3.0)[:, None]
    ref, lat = _run_both(op, lp, n, phi, u, 12)
    _fp32_bar(ref, lat, shape)
    assert lbm.lbm_tuning(lat.handle)["fd_tile_width"] == 1


def test_wave_kernel_cubic_at_half_and_f16(monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", "4,24,4,1,1")
    op, lp = _pair(128, 96, m=4, cubic_at_half=1, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.drop(2, 128, 96, R=24, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 128, 96)
    u = u + 0.003 * np.cos(np.arange(96) / 3.0)[None, :, None]
    ref, lat = _run_both(op, lp, n, phi, u, 15)
    _fp32_bar(ref, lat, "cubic_at_half")
    # FP16 deviation storage feeds the same FP32 phi and u* planes
    monkeypatch.setenv("HLBM_TUNING", "4,24,4,5,1")
    op, lp = _pair(128, 96, m=4, precision=lbm.LBM_F16DEV, **CFG1)
    ref, lat = _run_both(op, lp, n, phi, u, 12)
    dphi, du, _ = _errors(ref, lat)
    assert dphi <= 1e-3, dphi
    assert lbm.lbm_tuning(lat.handle)["fd_tile_width"] == 1


def test_wave_kernel_matches_block_kernel_spinodal(monkeypatch):
    """1024^2 spinodal state with a flow, 3 LB steps: the wavefront and the
    block FD kernels evaluate the same formulas with the same collide kernel;
    they may round differently (the block kernel's contraction is the
    compiler's), so they agree to FP32 round-off, not bitwise."""
    L = 1024
    phi = I.spinodal(2, L, L, seed=3)
    n, u = I.rest(2, L, L)
    u = u + 0.004 * np.sin(np.arange(L) / 7.0)[None, None, :]
    out = []
    for shape in ("4,96,2,5,128", "4,64,4,5,1", "2,64,4,5,1"):
        monkeypatch.setenv("HLBM_TUNING", shape)
        lat = lbm.Lattice(lbm.LbmParams(Lx=L, Ly=L, fd_substeps=4, precision=lbm.LBM_F32DEV, **CFG1))
        lat.init_fields(n, phi, u).step(3)
        out.append(lat.moments())
        lat.close()
    (n0, p0, u0), (n1, p1, u1), (n2, p2, u2) = out
    assert np.max(np.abs(p0 - p1)) <= 2e-7 and np.max(np.abs(u0 - u1)) <= 1e-8
    # four substeps in one launch or two launches of two: the wavefront kernel
    # evaluates the same explicitly rounded formulas in the same order
    assert np.array_equal(p1, p2) and np.array_equal(u1, u2)


@pytest.mark.parametrize("kw", [dict(adv_variant=1), dict(precision=lbm.LBM_F64)])
def test_wave_kernel_refused(kw, monkeypatch):
    """The wavefront kernel implements the printed advection form on FP32 phi:
    the flux form and the FP64 path are refused when it is requested."""
    monkeypatch.setenv("HLBM_TUNING", "4,32,4,1,1")
    args = dict(CFG1)
    args.update(kw)
    args.setdefault("precision", lbm.LBM_F32DEV)
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(lbm.LbmParams(Lx=128, Ly=64, **args))


def test_block_kernel_refused_in_fp64(monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", "4,80,2,1,128")
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(lbm.LbmParams(Lx=64, Ly=64, precision=lbm.LBM_F64, **CFG1))


@pytest.mark.parametrize("shape", ["4,16,4,2,0", "1,32,4,0,32", "2,32,4,0,64"])
def test_launch_shapes_flux_variant(shape, monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", shape)
    op, lp = _pair(64, 40, m=4, adv_variant=1, cubic_at_half=1, **CFG1)
    phi = I.drop(2, 64, 40, R=10, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 64, 40)
    u = u + 0.003 * np.cos(np.arange(40) / 3.0)[None, :, None]
    ref, lat = _run_both(op, lp, n, phi, u, 20)
    dphi, du, dn = _errors(ref, lat)
    assert dphi <= 1e-11 and du <= 1e-12 and dn <= 1e-11, (shape, dphi, du, dn)


# TMA-staged collide kernel (FP32, Lx % 4 == 0, sides >= 64): 3 scalar
# collision, 5 / 6 packed-pair collision budgeted for 4 / 3 CTAs per SM,
# 7 persistent and pipelined (32 x 16 tiles from a counter, two stages)
TMA_VARIANTS = [3, 5, 6, 7]


@pytest.mark.parametrize("variant", TMA_VARIANTS)
@pytest.mark.parametrize("size", [(64, 64), (100, 68), (300, 217)])
def test_tma_collide_against_oracle(variant, size, monkeypatch):
    """Every tile of 64 x 64 is an edge tile (the copies' zero-filled cells are
    all replaced by periodic images); 100 x 68 and 300 x 217 have ragged last
    tiles in both directions."""
    monkeypatch.setenv("HLBM_TUNING", f"4,80,2,{variant},128")
    Lx, Ly = size
    op, lp = _pair(Lx, Ly, m=4, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.drop(2, Lx, Ly, R=min(Lx, Ly) // 4, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, Lx, Ly)
    u = u + 0.003 * np.sin(np.arange(Lx) / 4.0)[None, None, :] + 0.002 * np.cos(np.arange(Ly) / 3.0)[None, :, None]
    ref, lat = _run_both(op, lp, n, phi, u, 12)
    _fp32_bar(ref, lat, (variant, size))
    assert lbm.lbm_tuning(lat.handle)["collide_sites_per_thread"] == variant


@pytest.mark.parametrize("variant", TMA_VARIANTS)
@pytest.mark.parametrize("extra", ["T", "force"])
def test_tma_collide_T_and_body_force(variant, extra, monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", f"4,80,2,{variant},128")
    kw = dict(CFG1)
    if extra == "T":
        kw["T"] = 0.28
    else:
        kw.update(g=(2e-5, -1e-5, 0.0), force_steps=6)
    op, lp = _pair(96, 72, m=4, precision=lbm.LBM_F32DEV, **kw)
    phi = I.drop(2, 96, 72, R=18, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, 96, 72)
    n = n + 0.001 * np.sin(np.arange(96) / 6.0)[None, :]
    ref, lat = _run_both(op, lp, n, phi, u, 12)
    _fp32_bar(ref, lat, (variant, extra))


@pytest.mark.parametrize("variant", TMA_VARIANTS)
def test_tma_collide_translation_equivariance_bitwise(variant, monkeypatch):
    """Shifting the initial state by whole tiles (32 sites) moves interior
    tiles onto the lattice's edges and back: the periodic images the edge
    CTAs reload must reproduce exactly what the copies deliver inside."""
    monkeypatch.setenv("HLBM_TUNING", f"4,80,2,{variant},128")
    op, lp = _pair(128, 96, precision=lbm.LBM_F32DEV, **CFG1)
    phi = I.spinodal(2, 128, 96, seed=5)
    n, u = I.rest(2, 128, 96)
    res = []
    for shift in ((0, 0), (32, 64)):
        lat = lbm.Lattice(lp)
        lat.init_fields(n, np.roll(phi, shift, axis=(0, 1)), u).step(60)
        res.append(lat.moments())
        lat.close()
    for a, b in zip(res[0], res[1]):
        axes = (0, 1) if a.ndim == 2 else (1, 2)
        assert np.array_equal(np.roll(a, (32, 64), axis=axes), b)


def test_tma_collide_refused_where_ineligible(monkeypatch):
    """Lx % 4 != 0 (a copy's rows must start on 16-byte boundaries), a side
    below 64, and FP64 storage are refused for the TMA kernel."""
    for Lx, Ly, prec in ((66, 64, lbm.LBM_F32DEV), (64, 48, lbm.LBM_F32DEV), (64, 64, lbm.LBM_F64)):
        monkeypatch.setenv("HLBM_TUNING", "4,16,2,3,0")
        with pytest.raises(lbm.LbmError):
            lbm.Lattice(lbm.LbmParams(Lx=Lx, Ly=Ly, precision=prec, **CFG1))


@pytest.mark.parametrize("gx", [1e-5, 3e-5, 5e-5])
def test_paper_drop_convection_full_size(gx):
    """Sec. III, Figs. 5-6 at the paper's size: a drop of diameter 64 on 256 x
    128 (-a = b = 1e-3, kappa = 3e-3, Gamma = 5, tau = 1, OC, dt_FD = dt_LB)
    pushed by G = n (g_x, 0) for t < 500 over the printed range of g_x, then
    free: the whole fluid moves at 500 g_x, the drop's centre of mass (Eq. 40)
    moves with the fluid velocity there (v_CM = v_f within 1 %), and its
    horizontal and vertical diameters stay within 3 % of each other."""
    Lx, Ly = 256, 128
    kw = dict(a=-1e-3, b=1e-3, kappa=3e-3, tau=1.0, Gamma=5.0, N=0.3, Q=2.5)
    op = O.Params(Lx=Lx, Ly=Ly, m=1, **kw)
    lp = lbm.LbmParams(Lx=Lx, Ly=Ly, g=(gx, 0.0, 0.0), force_steps=500, fd_substeps=1,
                       precision=lbm.LBM_F64, **kw)
    phi = I.drop(2, Lx, Ly, R=32, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, Lx, Ly)
    lat = lbm.Lattice(lp).init_fields(n, phi, u)
    lat.step(600)
    d = lat.diagnostics()
    xs, vfs = [d["r_cm"][0]], []
    for _ in range(4):
        lat.step(100)
        d = lat.diagnostics()
        xs.append(d["r_cm"][0])
        vfs.append(d["v_f"][0])
    v_cm = np.diff(xs) / 100.0
    gn, gphi, gu = lat.moments()
    lat.close()
    assert np.sum(gn * gu[0]) / np.sum(gn) == pytest.approx(500 * gx, rel=5e-3)
    np.testing.assert_allclose(np.mean(v_cm), np.mean(vfs), rtol=1e-2)
    cx, cy = d["r_cm"][0], d["r_cm"][1]

    def width(profile, c):
        prof = np.roll(profile, len(profile) // 2 - int(round(c)))
        s = np.sign(prof)
        idx = np.where(s[:-1] != s[1:])[0]
        zs = [i + prof[i] / (prof[i] - prof[i + 1]) for i in idx]
        return zs[-1] - zs[0]

    ratio = width(gphi[int(round(cy)) % Ly], cx) / width(gphi[:, int(round(cx)) % Lx], cy)
    print(f"g_x {gx}: v_CM {np.mean(v_cm):.4e}, v_f {np.mean(vfs):.4e}, diameter ratio {ratio:.4f}")
    assert abs(ratio - 1) < 0.03


@pytest.mark.parametrize("variant", [3, 5])
@pytest.mark.parametrize("size", [(64, 64), (104, 72), (304, 217)])
def test_tma_collide_fp16_storage(variant, size, monkeypatch):
    """FP16 deviations (scale 2^10) through the TMA kernel (copies of 32- and
    40-half boxes, 8-element x origins): against the FP16 register kernel,
    which stores the same FP16 values and differs only in the FP32
    arithmetic's order, and loosely against the FP64 oracle."""
    Lx, Ly = size
    op, _ = _pair(Lx, Ly, m=4, **CFG1)
    phi = I.drop(2, Lx, Ly, R=min(Lx, Ly) // 4, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(2, Lx, Ly)
    u = u + 0.003 * np.sin(np.arange(Lx) / 4.0)[None, None, :]
    res = {}
    for shape in (f"4,80,2,{variant},128", "4,80,2,2,128"):
        monkeypatch.setenv("HLBM_TUNING", shape)
        lat = lbm.Lattice(lbm.LbmParams(Lx=Lx, Ly=Ly, fd_substeps=-4, precision=lbm.LBM_F16DEV, **CFG1))
        lat.init_fields(n, phi, u).step(12)
        assert lbm.lbm_tuning(lat.handle)["collide_sites_per_thread"] == int(shape.split(",")[3])
        res[shape] = lat.moments()
        lat.close()
    a, b = res[f"4,80,2,{variant},128"], res["4,80,2,2,128"]
    ref = O.State.create(op, n, phi, u)
    ref.run(12)
    rn, ru = ref.moments()
    umax = float(np.max(np.sqrt(np.sum(ru * ru, axis=0))))
    assert np.max(np.abs(a[1] - b[1])) <= 1e-4
    assert np.max(np.abs(a[2] - b[2])) <= 2e-2 * umax
    assert np.max(np.abs(a[1] - ref.phi)) <= 1e-3
    assert np.max(np.abs(a[2] - ru)) <= 0.1 * umax


def test_tma_collide_fp16_translation_equivariance_bitwise(monkeypatch):
    monkeypatch.setenv("HLBM_TUNING", "4,80,2,5,128")
    lp = lbm.LbmParams(Lx=128, Ly=96, fd_substeps=-4, precision=lbm.LBM_F16DEV, **CFG1)
    phi = I.spinodal(2, 128, 96, seed=5)
    n, u = I.rest(2, 128, 96)
    res = []
    for shift in ((0, 0), (32, 64)):
        lat = lbm.Lattice(lp)
        lat.init_fields(n, np.roll(phi, shift, axis=(0, 1)), u).step(60)
        res.append(lat.moments())
        lat.close()
    for a, b in zip(res[0], res[1]):
        axes = (0, 1) if a.ndim == 2 else (1, 2)
        assert np.array_equal(np.roll(a, (32, 64), axis=axes), b)


def test_laplace_law_3d_drop_64():
    """The Laplace law in 3D (Eqs. 4, 6; reading c-xvi for the D3Q19
    stencils): the drop of radius 16 on 64^3 with the 3D workload's
    parameters (FP64 path, which equals the oracle to 1e-11), the pressure
    jump p0(centre) - p0(far corner) sampled every 10 steps over
    t = 500 ... 1500 (sound waves make single samples swing by +-40 %)
    averages to 2 sigma / R_eff within 6 % (the oracle gives 1.01)."""
    L = 64
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    op = O.Params(dims=3, Lx=L, Ly=L, Lz=L, m=8, **kw)
    lp = lbm.LbmParams(dims=3, Lx=L, Ly=L, Lz=L, fd_substeps=-8, precision=lbm.LBM_F64, **kw)
    phi = I.drop(3, L, L, L, R=16, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, L, L, L)
    lat = lbm.Lattice(lp).init_fields(n, phi, u)
    lat.step(500)
    dps = []
    for _ in range(100):
        lat.step(10)
        d = lat.diagnostics()
        dps.append(d["dp"])
    lat.close()
    laplace = 2 * O.sigma_of(op) / d["R_eff"]
    print(f"3D Laplace: <dp> = {np.mean(dps):.5e}, 2 sigma / R_eff = {laplace:.5e}, "
          f"ratio {np.mean(dps) / laplace:.4f}, R_eff {d['R_eff']:.3f}")
    np.testing.assert_allclose(np.mean(dps), laplace, rtol=0.06)
    assert d["u_max"] < 2e-3


def test_drop3d_full_size_sampled():
    """The 3D drop workload at its full size and in its benchmark launch
    configuration (256^3, R = 48, D3Q19, N = 1/6, Q = 1/3, m chosen by the
    library = 8, the fused fd3f FD kernel of Lx = 256), with a uniform flow
    (0.01, -0.005, 0.007) added so that advection acts along every axis:
    after one LB step, the 36^3 inner blocks of three 96^3 boxes (on the
    drop's interface along x and along z, and one wrapping around all three
    faces) against the oracle run on those boxes (sampled parity: the inner
    block is exact, tests/test_oracle_boxes.py).  FP32 deviations to the
    64^3 test's bar, FP16 deviations to theirs."""
    from sampling import box_oracle
    L, W, steps = 256, 96, 1
    kw = dict(CFG1, N=1 / 6, Q=1 / 3)
    op = O.Params(dims=3, Lx=L, Ly=L, Lz=L, m=8, **kw)
    phi = I.drop(3, L, L, L, R=48, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(3, L, L, L)
    for k, v in enumerate((0.01, -0.005, 0.007)):
        u[k] += v
    boxes = [box_oracle(dict(kw, m=8), n, phi, u, c, W, steps)
             for c in ((128, 128, 176), (80, 128, 128), (2, 250, 5))]  # (z, y, x)
    for prec, bphi, bu in ((lbm.LBM_F32DEV, 1e-5, 1e-3), (lbm.LBM_F16DEV, 1e-2, 0.2)):
        lat = lbm.Lattice(lbm.LbmParams(dims=3, Lx=L, Ly=L, Lz=L, precision=prec, **kw))
        assert lat.m == 8
        lat.init_fields(n, phi, u).step(steps)
        gn, gphi, gu = lat.moments()
        lat.close()
        for inner, rn, rphi, ru in boxes:
            ix = np.ix_(*inner)
            dphi = float(np.max(np.abs(gphi[ix] - rphi)))
            du = float(np.max(np.abs(np.stack([gu[k][ix] for k in range(3)]) - ru)))
            dn = float(np.max(np.abs(gn[ix] - rn)))
            umax = float(np.max(np.abs(ru)))
            print(f"256^3 sampled, precision {prec}: |dphi|={dphi:.3e} |du|={du:.3e} "
                  f"|dn|={dn:.3e} umax={umax:.3e}")
            assert dphi <= bphi and du <= bu * umax and dn <= 10 * bphi, (prec, dphi, du, dn)


def test_spinodal_4096_sampled():
    """The 4096^2 lines of the benchmark (the size where the collide kernel is
    HBM-bound), FP32 and FP16 deviations in the autotuned launch
    configuration the benchmark uses (m = 4): the workload's spinodal
    initial state with a flow 0.003 sin(x/4) added so that u* is not
    vanishingly small, three LB steps, then the 52^2 inner blocks of four
    160^2 boxes (one wrapping around both faces) against the oracle on those
    boxes (sampled parity; tests/test_oracle_boxes.py)."""
    from sampling import box_oracle
    L, W, steps, m = 4096, 160, 3, 4
    phi = I.spinodal(2, L, L, seed=0)
    n, u = I.rest(2, L, L)
    u = u + 0.003 * np.sin(np.arange(L) / 4.0)[None, None, :]
    boxes = [box_oracle(dict(CFG1, m=m), n, phi, u, c, W, steps)
             for c in ((2048, 2048), (100, 3000), (4000, 17), (3, 4093))]  # (y, x)
    for prec, bphi, bu in ((lbm.LBM_F32DEV, 1e-6, 1e-3), (lbm.LBM_F16DEV, 1e-3, 0.1)):
        lat = lbm.Lattice(lbm.LbmParams(Lx=L, Ly=L, fd_substeps=m, precision=prec, **CFG1))
        lat.init_fields(n, phi, u).step(steps)
        tuning = lbm.lbm_tuning(lat.handle)
        gn, gphi, gu = lat.moments()
        lat.close()
        for inner, rn, rphi, ru in boxes:
            ix = np.ix_(*inner)
            dphi = float(np.max(np.abs(gphi[ix] - rphi)))
            du = float(np.max(np.abs(np.stack([gu[k][ix] for k in range(2)]) - ru)))
            dn = float(np.max(np.abs(gn[ix] - rn)))
            umax = float(np.max(np.abs(ru)))
            print(f"4096^2 sampled, precision {prec}, tuning {tuning}: |dphi|={dphi:.3e} "
                  f"|du|={du:.3e} |dn|={dn:.3e} umax={umax:.3e}")
            assert dphi <= bphi and du <= bu * umax and dn <= 10 * bphi, (prec, dphi, du, dn)
