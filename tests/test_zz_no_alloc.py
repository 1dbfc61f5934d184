"""The allocation-free prefilter entry point (mreg_prefilter_noalloc).

It serves callers that cannot call cudaMalloc (hosts whose own memory pool
owns all device memory, loops that must not pay for a device-synchronising
allocation).  It must give the same B-spline coefficients as the
regular set-up path (mreg_create, read back with mreg_get_field), on two calls
in a row that share its fixed scratch array.  This file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

from oracle import bspline

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mreg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_2141_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    from paper_1411_2141_gb300 import mreg as m
    m.load()
    return m


def _image(H, W, seed):
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    return (np.sin(xs / 5.3) * np.cos(ys / 3.7) + 0.2 * rng.normal(size=(H, W))).astype(np.float32)


def _reference_coefficients(mreg, img):
    """Coefficients from the regular path: mreg_create prefilters Te."""
    H, W = img.shape
    V = np.array([[0, 0], [W - 1, 0], [W - 1, H - 1], [0, H - 1]], np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    with mreg.Registration(V, T, img, img, 0.1, 1.0) as r:
        return r.get_field(mreg.MREG_FIELD_COEF_TE)


def test_noalloc_prefilter_matches_create_path_twice(mreg):
    shapes = [(300, 257), (512, 512)]
    for k, (H, W) in enumerate(shapes):   # two calls in a row on the shared scratch
        img = _image(H, W, seed=k)
        ref = _reference_coefficients(mreg, img)
        # strided device input: a view into a wider tensor
        big = torch.zeros((H, W + 5), dtype=torch.float32, device="cuda")
        big[:, :W] = torch.from_numpy(img)
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        mreg.prefilter_noalloc(big[:, :W], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        tol = 5e-6 * np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol
        # and against the FP64 oracle, with the same tolerance
        assert np.abs(got - bspline.prefilter_2d(img)).max() <= tol


def test_noalloc_prefilter_rejects_oversized_images(mreg):
    img = torch.zeros((1025, 1024), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(img)
    with pytest.raises(mreg.MregError) as e:
        mreg.prefilter_noalloc(img, out)
    assert e.value.status == mreg.MREG_ERR_INVALID_ARG
    assert "MREG_NOALLOC_MAX_PIXELS" in str(e.value)


def test_noalloc_prefilter_rejects_memory_the_gpu_cannot_use(mreg):
    H, W = 64, 48
    out = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):   # the binding refuses CPU tensors
        mreg.prefilter_noalloc(torch.zeros((H, W), dtype=torch.float32), out)
    with pytest.raises(ValueError):
        mreg.prefilter_noalloc(out, torch.zeros((H, W), dtype=torch.float32))
    # the C entry point itself refuses a host address before launching anything
    host = np.zeros((H, W), np.float32)
    lib = mreg.load()
    assert lib.mreg_prefilter_noalloc(host.ctypes.data, W, out.data_ptr(), W, H,
                                      None) == mreg.MREG_ERR_INVALID_ARG
    assert b"device memory" in lib.mreg_last_error()
    assert lib.mreg_prefilter_noalloc(out.data_ptr(), W, host.ctypes.data, W, H,
                                      None) == mreg.MREG_ERR_INVALID_ARG
    # and a valid call afterwards still works
    img = torch.from_numpy(_image(H, W, seed=7)).cuda()
    mreg.prefilter_noalloc(img, out)
    torch.cuda.synchronize()
    ref = bspline.prefilter_2d(img.cpu().numpy())
    assert np.abs(out.cpu().numpy() - ref).max() <= 5e-6 * np.abs(ref).max()
