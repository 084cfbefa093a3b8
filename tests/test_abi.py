"""CPU checks of the C ABI: the library builds, loads and exports every symbol
declared in include/hybrid_lbm.h; parameter validation runs before any CUDA
call, so invalid parameters give LBM_EINVAL with a message even without a GPU.
"""
import ctypes
import os
import re

import pytest

from paper_0902_3921_gb300 import build as B
from paper_0902_3921_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.load_library()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert "lbm_create" in declared and "lbm_step" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(lbm.EXPORTS) <= declared


def test_struct_layouts_match_header():
    # the ctypes mirrors must match the C structs field for field
    src = open(os.path.join(ROOT, "include", "hybrid_lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for name, mirror in (("lbm_params", lbm.c_lbm_params), ("lbm_diag", lbm.c_lbm_diag),
                         ("lbm_buffers", lbm.c_lbm_buffers)):
        seg = [s for s in src.split("typedef struct {") if ("} " + name + ";") in s][0]
        body = seg.split("} " + name + ";")[0]
        fields = re.findall(r"(\w+)(?:\[\d\])?\s*[;,]", body)
        assert [f for f, _ in mirror._fields_] == fields, name
        assert ctypes.sizeof(mirror) % 8 == 0


def test_lattice_tables(lib):
    import numpy as np
    for dims, q in ((2, 9), (3, 19)):
        e, w = lbm.lbm_lattice(dims)
        assert e.shape == (q, 3)
        assert abs(w.sum() - 1) < 1e-15
        np.testing.assert_allclose(w @ e, 0, atol=1e-16)
    assert lib.lbm_lattice(4, None, None) == lbm.LBM_EINVAL


@pytest.mark.parametrize("change,needle", [
    (dict(tau=0.5), "tau"),
    (dict(b=0.0), "b must"),
    (dict(kappa=-1.0), "kappa"),
    (dict(Gamma=-1.0), "Gamma"),
    (dict(Lx=2), ">= 3"),
    (dict(dims=4), "dims"),
    (dict(precision=7), "precision"),
    (dict(adv_variant=3), "adv_variant"),
    (dict(fd_substeps=1), "Euler bound"),
    (dict(N=float("nan")), "finite"),
    (dict(T=0.0), "T > 0"),
    (dict(force_steps=-1), "force_steps"),
    (dict(f16_scale_log2=20), "f16_scale_log2"),
    (dict(dims=3, Lx=2048, Ly=2048, Lz=1024), "2^31"),
    (dict(fd_substeps=-5000), "fd_substeps too large"),
    (dict(g=(float("inf"), 0.0, 0.0)), "g must be finite"),
    (dict(a=float("nan")), "a must be finite"),
])
def test_invalid_parameters_are_rejected(lib, change, needle):
    p = lbm.LbmParams(**change)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(p)
    assert ei.value.code == lbm.LBM_EINVAL
    assert needle in str(ei.value)


def test_null_handle_calls_are_safe(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_synchronize(None) == lbm.LBM_EINVAL
    assert lib.lbm_time(None) == -1
    lib.lbm_free(None)
    assert lib.lbm_create(None, None, None) == lbm.LBM_EINVAL


def test_fd_substep_rule():
    """Sec. II C: dt_LB = m dt_FD.  The default m is the smallest with the
    diffusive stiffness Gamma (a_eff lam + kappa lam^2) * dt <= 1.5; an
    explicit m below the Euler bound (<= 2) is refused unless forced (m < 0).
    Checked on the host-side arithmetic through the error text."""
    # the drop configuration: stiffness 5.28 in 2D -> m_min = 3
    with pytest.raises(lbm.LbmError, match="m >= 3"):
        lbm.lbm_create(lbm.LbmParams(fd_substeps=2))
    with pytest.raises(lbm.LbmError, match="m >= 6"):
        lbm.lbm_create(lbm.LbmParams(dims=3, Lz=8, fd_substeps=5))


def test_buffer_bytes_and_adoption_checks(lib):
    """lbm_buffer_bytes is arithmetic on the parameters; lbm_create_with_buffers
    refuses NULL or unaligned buffers before touching CUDA."""
    kw = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5)
    S2 = 64 * 48
    assert lbm.lbm_buffer_bytes(lbm.LbmParams(Lx=64, Ly=48, precision=lbm.LBM_F32DEV, **kw)) == (
        9 * 4 * S2, 4 * S2, 2 * 4 * S2)
    assert lbm.lbm_buffer_bytes(lbm.LbmParams(Lx=64, Ly=48, precision=lbm.LBM_F64, **kw)) == (
        9 * 8 * S2, 8 * S2, 2 * 8 * S2)
    S3 = 10 * 12 * 14
    assert lbm.lbm_buffer_bytes(lbm.LbmParams(dims=3, Lx=10, Ly=12, Lz=14, precision=lbm.LBM_F16DEV,
                                              **kw)) == (19 * 2 * S3, 4 * S3, 3 * 4 * S3)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_buffer_bytes(lbm.LbmParams(Lx=64, Ly=48, **dict(kw, tau=0.4)))
    p = lbm.LbmParams(Lx=64, Ly=48, precision=lbm.LBM_F32DEV, **kw)
    for pops, phi, u in (([0, 4096], [4096] * 3, 4096), ([4096, 4096], [4096, 4100, 4096], 4096)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create_with_buffers(p, pops, phi, u)
        assert e.value.code == lbm.LBM_EINVAL


def _prototypes():
    """name -> (return type, [parameter types]) of every function declared in
    include/*.h (comments stripped; parameter names dropped)."""
    protos = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for ret, name, params in re.findall(r"([\w\s\*]+?)\b(lbm_\w+)\s*\(([^)]*)\)\s*;", src):
            ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
            types = []
            for p_ in ps:
                is_ptr = "*" in p_ or "[" in p_
                words = re.sub(r"\[\d*\]", "", p_).replace("*", " ").split()
                base = " ".join(w for w in words[:-1] if w != "const") if len(words) > 1 else words[0]
                types.append("ptr" if is_ptr else base)
            r = ret.replace("const", "").split()
            protos[name] = ("ptr" if "*" in ret else " ".join(r[-3:]).strip(), types)
    return protos


_SCALAR = {"int": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float,
           "long long": ctypes.c_longlong, "unsigned long long": ctypes.c_ulonglong}


def _is_pointer_type(t):
    return (t in (ctypes.c_void_p, ctypes.c_char_p) or isinstance(t, type(ctypes.POINTER(ctypes.c_int)))
            or hasattr(t, "from_param") and t not in _SCALAR.values())


def test_binding_argtypes_match_prototypes(lib):
    """Every binding that declares argtypes has one per C parameter, scalars
    of the C type and pointers where the C side takes a pointer; restypes of
    the functions that do not return int match too."""
    protos = _prototypes()
    assert len(protos) >= 40
    checked = 0
    for name, (ret, params) in protos.items():
        f = getattr(lib, name)
        at = getattr(f, "argtypes", None)
        if at is None:
            continue
        checked += 1
        assert len(at) == len(params), (name, len(at), params)
        for i, (c, t) in enumerate(zip(params, at)):
            if c == "ptr":
                assert _is_pointer_type(t), (name, i, t)
            else:
                assert t is _SCALAR[c.replace("const ", "")], (name, i, c, t)
        if ret == "ptr":
            assert f.restype in (ctypes.c_char_p, ctypes.c_void_p), (name, f.restype)
        elif ret in ("long long", "unsigned long long", "double", "float"):
            assert f.restype is _SCALAR[ret], (name, ret, f.restype)
        elif ret == "void":
            assert f.restype is None, (name, f.restype)
    assert checked >= 30


_OK_INST = (32, 48, (0.0, 0.0), 0)


@pytest.mark.parametrize("common,instances,needle", [
    (dict(dims=3), [_OK_INST], "batches are 2D"),
    (dict(precision=lbm.LBM_F16DEV), [_OK_INST], "FP64 or FP32-deviation"),
    (dict(T=0.25), [_OK_INST], "T = 1/3"),
    (dict(tau=0.5), [_OK_INST], "bad common parameters"),
    (dict(adv_variant=7), [_OK_INST], "adv_variant"),
    (dict(fd_substeps=1), [_OK_INST], "Euler bound"),
    (dict(), [_OK_INST, (2, 48, (0.0, 0.0), 0)], "bad instance 1"),
    (dict(), [_OK_INST, _OK_INST, (32, 32, (float("nan"), 0.0), 0)], "bad instance 2"),
    (dict(), [(32, 32, (0.0, 0.0), -5)], "bad instance 0"),
    (dict(), [], "NULL or empty batch"),
])
def test_invalid_batches_are_rejected(lib, common, instances, needle):
    """lbm_batch_create validates its parameters and every instance before
    any CUDA call: EINVAL with the reason, no handle."""
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Batch(lbm.LbmParams(**common), instances)
    assert ei.value.code == lbm.LBM_EINVAL
    assert needle in str(ei.value)


@pytest.mark.parametrize("channels,layers", [(24, 6), (32, 1), (16, 9)])
def test_invalid_networks_are_rejected(lib, channels, layers):
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Net(channels, layers)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "channels must be 16 or 32" in str(ei.value)


NOALLOC_BAD = [
    (dict(dims=4), "dims"),
    (dict(Lx=2), "side"),
    (dict(a=float("nan")), "a must be"),
    (dict(a=0.05), "a must be"),
    (dict(b=0.0), "b must be"),
    (dict(kappa=float("inf")), "kappa"),
    (dict(kappa=-1.0), "kappa"),
    (dict(T=0.0), "T must be"),
    (dict(T=float("nan")), "T must be"),
    (dict(N=float("nan")), "N and Q"),
    (dict(Q=float("inf")), "N and Q"),
    # one site beyond the scratch capacity (4194305 = 838861 x 5)
    (dict(Lx=838861, Ly=5), "capacity"),
]


@pytest.mark.parametrize("bad,why", NOALLOC_BAD)
def test_noalloc_refuses_invalid_parameters_before_any_cuda_call(lib, bad, why):
    """lbm_diagnostics_noalloc checks the fields it reads as lbm_create does,
    and its site capacity, before touching the GPU (none is needed here)."""
    kw = dict(Lx=64, Ly=64, a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
    kw.update(bad)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_diagnostics_noalloc(lbm.LbmParams(**kw), 1 << 20)
    assert ei.value.code == lbm.LBM_EINVAL
    assert why in str(ei.value), str(ei.value)


def test_noalloc_capacity_is_exactly_the_declared_maximum(lib):
    """A lattice of exactly LBM_NOALLOC_MAX_SITES sites passes every check
    before the CUDA calls (without a GPU the call then fails with ECUDA, not
    EINVAL); one site more is refused."""
    src = open(os.path.join(ROOT, "include", "hybrid_lbm.h")).read()
    assert "#define LBM_NOALLOC_MAX_BLOCKS 2048" in src
    assert "#define LBM_NOALLOC_MAX_SITES (LBM_NOALLOC_MAX_BLOCKS * 2048)" in src
    import torch
    if torch.cuda.is_available():
        pytest.skip("the ECUDA branch needs a machine without a GPU")
    kw = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_diagnostics_noalloc(lbm.LbmParams(Lx=2048, Ly=2048, **kw), 1 << 20)
    assert ei.value.code == lbm.LBM_ECUDA


def test_injected_allocation_fault_is_refused_before_any_cuda_call(lib, monkeypatch):
    """LBM_FAULT=alloc: lbm_create reports LBM_ENOMEM as if the first device
    allocation failed, before it touches the GPU (none is needed here)."""
    monkeypatch.setenv("LBM_FAULT", "alloc")
    kw = dict(Lx=64, Ly=64, a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice(lbm.LbmParams(**kw))
    assert ei.value.code == lbm.LBM_ENOMEM
    assert "injected fault" in str(ei.value)


@pytest.mark.parametrize("bad", [dict(stencil_fd=2), dict(stencil_fd=1, dims=3, Lz=8, N=1 / 6, Q=1 / 3),
                                 dict(stencil_fd=1, adv_variant=1), dict(stencil_fd=1, Q=-0.5)])
def test_stencil_fd_refusals_before_any_cuda_call(lib, bad):
    """stencil_fd is 0 or 1, 2D only, and only with the printed advection form
    (the paper defines no stencil for the upwind fluxes)."""
    kw = dict(Lx=64, Ly=64, a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
    kw.update(bad)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice(lbm.LbmParams(**kw))
    assert ei.value.code == lbm.LBM_EINVAL and "stencil_fd" in str(ei.value)
