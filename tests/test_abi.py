"""The C ABI library: builds for sm_103a, loads, exports every function that
include/mreg.h declares, and rejects bad arguments on the host side (these
checks run before any CUDA call, so they need no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1411_2141_gb300 import build as build_mod
from paper_1411_2141_gb300 import mreg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return mreg.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "mreg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mreg_[a-z_]+)\s*\(", text)))


def test_exports_match_header(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(mreg.EXPORTS) == names


def test_version_and_defaults(lib):
    assert lib.mreg_version() == 1
    o = mreg.default_options()
    assert (o.mode, o.grad, o.quad, o.pcg_maxit) == (0, 0, 0, 100)
    assert o.lambda_ < 0 and o.pcg_rtol == 1e-7


def _mesh_square(W=8, H=6):
    V = np.array([[0, 0], [W - 1, 0], [W - 1, H - 1], [0, H - 1]], np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return V, T


def _create(V, T, Re, Te, alpha=0.1, tau=1.0, **kw):
    return mreg.Registration(V, T, Re, Te, alpha, tau, **kw)


def _expect(status, fn):
    with pytest.raises(mreg.MregError) as e:
        fn()
    assert e.value.status == status, str(e.value)
    return str(e.value)


def test_host_validation_errors(lib):
    V, T = _mesh_square()
    img = np.zeros((6, 8), np.float32)
    E = mreg
    _expect(E.MREG_ERR_SIZE_MISMATCH, lambda: _create(V, T, img, np.zeros((6, 9), np.float32)))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, np.zeros((1, 8), np.float32),
                                                    np.zeros((1, 8), np.float32)))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, alpha=-1.0))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, tau=0.0))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode=7))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S1", quad="Q1"))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, pcg_rtol=0.0))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, pcg_maxit=0))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, block_size=100))
    bad = T.copy()
    bad[1, 2] = 9
    _expect(E.MREG_ERR_BAD_MESH, lambda: _create(V, bad, img, img))
    out = V.copy()
    out[2] = [7.5, 5.0]
    _expect(E.MREG_ERR_BAD_MESH, lambda: _create(out, T, img, img))
    flat = np.array([[0, 0], [7, 0], [3.5, 0], [0, 5]], np.float32)
    _expect(E.MREG_ERR_BAD_MESH, lambda: _create(flat, np.array([[0, 1, 2], [0, 1, 3]], np.int32), img, img))
    msg = _expect(E.MREG_ERR_BAD_MESH, lambda: _create(V, T[:1], img, img))
    assert "tile" in msg
    nan = img.copy()
    nan[2, 3] = np.nan
    _expect(E.MREG_ERR_NONFINITE, lambda: _create(V, T, nan, img))
    Vn = V.copy()
    Vn[0, 0] = np.inf
    _expect(E.MREG_ERR_NONFINITE, lambda: _create(Vn, T, img, img))


def test_raw_abi_null_arguments(lib):
    h = C.c_void_p()
    assert lib.mreg_create(None, None, None, 0.1, 1.0, None, None, C.byref(h)) == mreg.MREG_ERR_INVALID_ARG
    assert h.value is None
    assert lib.mreg_step(None, 1, None) == mreg.MREG_ERR_INVALID_ARG
    assert lib.mreg_default_options(None) == mreg.MREG_ERR_INVALID_ARG
    assert b"NULL" in lib.mreg_last_error()
    lib.mreg_destroy(None)


def test_clockwise_triangles_are_accepted_until_device_setup(lib):
    """A clockwise mesh passes host validation; without a GPU the call then
    fails cleanly with a CUDA status instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("covered by the GPU tests")
    V, T = _mesh_square()
    img = np.zeros((6, 8), np.float32)
    _expect(mreg.MREG_ERR_CUDA, lambda: _create(V, T[:, [0, 2, 1]], img, img))


def test_batch_host_validation_errors(lib):
    """Argument errors of the batched engine are found before any CUDA call
    and name the failing pair."""
    V, T = _mesh_square()
    img = np.zeros((6, 8), np.float32)
    E = mreg
    good = (V, T, img, img)
    _expect(E.MREG_ERR_SIZE_MISMATCH,
            lambda: mreg.Batch([good, (V, T, img, np.zeros((6, 9), np.float32))], 0.1, 1.0))
    with pytest.raises(mreg.MregError, match="pair 2"):
        mreg.Batch([good, good, (V, T, img, np.zeros((6, 9), np.float32))], 0.1, 1.0)
    _expect(E.MREG_ERR_INVALID_ARG, lambda: mreg.Batch([good], 0.1, 1.0, team_ctas=3))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: mreg.Batch([good], -0.1, 1.0))
    _expect(E.MREG_ERR_BAD_MESH,
            lambda: mreg.Batch([good, (V, np.array([[0, 1, 9]], np.int32), img, img)], 0.1, 1.0))
    h = C.c_void_p()
    assert lib.mreg_batch_create(0, None, None, None, 0.1, 1.0, None, None,
                                 C.byref(h)) == mreg.MREG_ERR_INVALID_ARG
    assert lib.mreg_batch_run(None, 1, None) == mreg.MREG_ERR_INVALID_ARG
    lib.mreg_batch_destroy(None)


def test_option_validation_of_the_newer_fields(lib):
    V, T = _mesh_square()
    img = np.zeros((6, 8), np.float32)
    E = mreg
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, smooth_passes=-1))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, smooth_passes=65))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S1", smooth_passes=2))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, team_blocks_per_sm=3))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S1", node_lanes=3))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S0", node_lanes=2))
    _expect(E.MREG_ERR_INVALID_ARG,
            lambda: _create(V, T, img, img, mode="S1", node_lanes=2, team_blocks_per_sm=2))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, engine=2))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S1", solver=3))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S2", grad="G1",
                                                    solver="chebyshev"))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: _create(V, T, img, img, mode="S0",
                                                    solver="chebyshev"))
    _expect(E.MREG_ERR_INVALID_ARG, lambda: mreg.Batch([(V, T, img, img)], 0.1, 1.0, mode="S1",
                                                       node_lanes=2))
    o = mreg.make_options(host_topology=True)
    assert o.host_topology == 1
    o.host_topology = 2
    h = C.c_void_p()
    im = mreg._image(img, [])
    mesh = mreg.mreg_mesh(4, 2, V.ctypes.data_as(C.POINTER(C.c_float)),
                          T.ctypes.data_as(C.POINTER(C.c_int32)))
    assert lib.mreg_create(C.byref(mesh), C.byref(im), C.byref(im), 0.1, 1.0, C.byref(o), None,
                           C.byref(h)) == mreg.MREG_ERR_INVALID_ARG
    o = mreg.make_options(coeff_bf16=True)
    assert o.coeff_storage == mreg.MREG_COEFF_BF16
    assert mreg.make_options(coeff="fp16").coeff_storage == mreg.MREG_COEFF_FP16
    o.coeff_storage = 3
    assert lib.mreg_create(C.byref(mesh), C.byref(im), C.byref(im), 0.1, 1.0, C.byref(o), None,
                           C.byref(h)) == mreg.MREG_ERR_INVALID_ARG
    assert lib.mreg_warp_energy_grad(None, None, None, None, None) == mreg.MREG_ERR_INVALID_ARG
    assert lib.mreg_unroll_grad(None, None, 3, None, None, None) == mreg.MREG_ERR_INVALID_ARG


def test_options_struct_matches_the_header():
    """Every mreg_options field of the header is in the binding's struct, in order."""
    import re
    text = open(os.path.join(ROOT, "include", "mreg.h")).read()
    body = text[text.index("typedef struct {\n  int32_t mode;"):text.index("} mreg_options;")]
    names = [m.group(1) or m.group(2) for m in re.finditer(
        r"^\s*(?:(?:int32_t|double|void\*)\s+(\w+);|void\*?\s*\(\*(\w+)\))", body, flags=re.M)]
    assert [n if n != "lambda" else "lambda_" for n in names] == \
        [f for f, _ in mreg.mreg_options._fields_]


def test_stats_struct_matches_the_header():
    """Every mreg_stats_t field of the header is in the binding's struct, in order."""
    import re
    text = open(os.path.join(ROOT, "include", "mreg.h")).read()
    body = text[text.index("typedef struct {\n  int32_t iterations_done;"):text.index("} mreg_stats_t;")]
    names = re.findall(r"^\s*(?:int32_t|double)\s+(\w+);", body, flags=re.M)
    assert names == [f for f, _ in mreg.mreg_stats_t._fields_]
