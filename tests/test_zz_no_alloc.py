"""The allocation-free diagnostics entry point, lbm_diagnostics_noalloc.

It serves callers that cannot allocate device memory (a host framework that
owns all device memory through its own allocator, or a time-critical loop
where cudaMalloc/cudaFree would synchronise the device): its scratch lives in
a static device array.  This test calls it through the C ABI on device
fields that the test itself owns and checks it against lbm_diagnostics on the
same state, twice in a row.  It sits in its own file so that pytest collects
it last.
"""
import numpy as np
import pytest

from paper_0902_3921_gb300 import inputs as I
from paper_0902_3921_gb300 import lbm

pytestmark = pytest.mark.gpu

CFG1 = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
KEYS = ("sum_n", "sum_phi", "u_max", "dp", "area", "R_eff")


def _device_fields(lat):
    import torch
    n, phi, u = lat.moments()
    host = np.concatenate([n.reshape(-1), phi.reshape(-1), u.reshape(-1)])
    return torch.from_numpy(host).cuda()


def _compare(a, b):
    for k in KEYS:
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-13), k
    for k in ("momentum", "r_cm", "v_f"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-13)
    assert a["nonfinite"] == b["nonfinite"]


@pytest.mark.parametrize("dims,shape,prec", [(2, (64, 64), lbm.LBM_F64),
                                             (2, (200, 150), lbm.LBM_F32DEV),
                                             (3, (24, 20, 18), lbm.LBM_F64)])
def test_noalloc_matches_lbm_diagnostics_twice(dims, shape, prec):
    import torch
    from paper_0902_3921_gb300 import build as B
    B.build()
    lbm.load_library()
    if dims == 2:
        Lx, Ly = shape
        p = lbm.LbmParams(Lx=Lx, Ly=Ly, precision=prec, fd_substeps=4, **CFG1)
        phi = I.drop(2, Lx, Ly, R=Ly / 4, phi0=1.0, xi=np.sqrt(2.8))
        n, u = I.rest(2, Lx, Ly)
    else:
        Lx, Ly, Lz = shape
        p = lbm.LbmParams(dims=3, Lx=Lx, Ly=Ly, Lz=Lz, precision=prec, fd_substeps=8,
                          **dict(CFG1, N=1 / 6, Q=1 / 3))
        phi = I.drop(3, Lx, Ly, Lz, R=5, phi0=1.0, xi=np.sqrt(2.8))
        n, u = I.rest(3, Lx, Ly, Lz)
    lat = lbm.Lattice(p)
    lat.init_fields(n, phi, u).step(60)
    centre = [Lx / 2.0, Ly / 2.0, (Lz / 2.0 if dims == 3 else 0.0)]
    ref1 = lat.diagnostics()  # unwraps around the box centre
    f1 = _device_fields(lat)
    torch.cuda.synchronize()
    rc, got1 = lbm.lbm_diagnostics_noalloc(p, f1.data_ptr(), r_ref=centre)
    assert rc == lbm.LBM_OK
    _compare(got1, ref1)
    # a second call in a row, on a later state, unwrapping around the last r_cm
    lat.step(40)
    ref2 = lat.diagnostics()
    f2 = _device_fields(lat)
    torch.cuda.synchronize()
    rc, got2 = lbm.lbm_diagnostics_noalloc(p, f2.data_ptr(), r_ref=ref1["r_cm"])
    assert rc == lbm.LBM_OK
    _compare(got2, ref2)
    assert got2["sum_phi"] != got1["sum_phi"]
    lat.close()


def test_noalloc_at_full_capacity():
    """Exactly LBM_NOALLOC_MAX_SITES sites (2048 x 2048): every block row of
    the partial sums and the result vector stored right after them are used,
    where an off-by-one in their offsets would show; compared with
    lbm_diagnostics on the same state."""
    import torch
    from paper_0902_3921_gb300 import build as B
    B.build()
    lbm.load_library()
    L = 2048
    assert L * L == 2048 * 2048  # LBM_NOALLOC_MAX_SITES
    p = lbm.LbmParams(Lx=L, Ly=L, precision=lbm.LBM_F32DEV, fd_substeps=4, **CFG1)
    phi = I.drop(2, L, L, R=300, phi0=1.0, xi=np.sqrt(2.8))
    n, u = I.rest(2, L, L)
    u = u + 0.002 * np.sin(np.arange(L) / 9.0)[None, None, :]
    lat = lbm.Lattice(p)
    lat.init_fields(n, phi, u).step(10)
    ref = lat.diagnostics()
    f = _device_fields(lat)
    torch.cuda.synchronize()
    for _ in range(2):
        rc, got = lbm.lbm_diagnostics_noalloc(p, f.data_ptr(), r_ref=[L / 2.0, L / 2.0, 0.0])
        assert rc == lbm.LBM_OK
        _compare(got, ref)
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    lbm.load_library()
    p = lbm.LbmParams(Lx=838861, Ly=5, **CFG1)  # 4194305 sites: the capacity plus one
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_diagnostics_noalloc(p, 1 << 20)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "capacity" in str(ei.value)
