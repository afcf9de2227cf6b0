"""The library's FP32 <-> FP64 conversions on the integer pipe (gm_convert)
against the hardware / numpy conversions: FP32 -> FP64 must be exact
(bit-identical to the widening conversion) for normals, subnormals, signed
zeros and infinities; FP64 -> FP32 must truncate toward zero (numpy's
round-to-nearest result, stepped one ulp toward zero where it rounded away).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2007_12273_gb300 import build, gm as gm_
    build.build()
    gm_.load()
    return gm_


def test_f32_to_f64_exact(gm):
    rng = np.random.default_rng(3)
    bits = np.concatenate([
        rng.integers(0, 2 ** 32, 200000, dtype=np.uint64),           # every class, both signs
        np.arange(1, 4096, dtype=np.uint64),                           # small subnormals
        0x7FFFFF - np.arange(0, 4096, dtype=np.uint64),                # large subnormals
        np.array([0, 0x80000000, 0x7F800000, 0xFF800000, 0x00800000, 0x7F7FFFFF,
                  0x3F800000, 0xBF800000, 0x80000001, 0x807FFFFF], dtype=np.uint64),
    ]).astype(np.uint32)
    f = bits.view(np.float32)
    out = gm.gm_convert(torch.from_numpy(f).cuda()).cpu().numpy()
    ref = f.astype(np.float64)
    nan = np.isnan(f)
    assert np.array_equal(out[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    assert np.all(np.isnan(out[nan]))


def trunc_ref(d):
    """FP64 -> FP32 toward zero: the nearest FP32, moved one step toward
    zero where it is larger in magnitude than d; 2^128 and up (and
    infinities) become infinities"""
    with np.errstate(over="ignore"):
        f = d.astype(np.float32)
    away = np.abs(f.astype(np.float64)) > np.abs(d)
    f = np.where(away, np.nextafter(f, np.float32(0.0)), f).astype(np.float32)
    big = np.abs(d) >= 2.0 ** 128
    return np.where(big, np.copysign(np.float32(np.inf), d).astype(np.float32), f).astype(np.float32)


def test_f64_to_f32_truncates(gm):
    rng = np.random.default_rng(4)
    e = rng.integers(-160, 140, 300000)
    d = np.ldexp(rng.uniform(1.0, 2.0, e.size), e) * rng.choice([-1.0, 1.0], e.size)
    d = np.concatenate([
        d,
        rng.uniform(-1, 1, 20000),
        np.ldexp(rng.uniform(1.0, 2.0, 20000), rng.integers(-150, -125, 20000)),  # FP32 subnormal range
        np.array([0.0, -0.0, np.inf, -np.inf, 2.0 ** 128, -2.0 ** 128, np.finfo(np.float32).max,
                  np.nextafter(2.0 ** 128, 0.0), 2.0 ** -149, 2.0 ** -150, 5e-324, 1.0, -1.0,
                  np.float64(np.float32(0.1))]),
    ])
    out = gm.gm_convert(torch.from_numpy(d).cuda()).cpu().numpy()
    ref = trunc_ref(d)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32)), \
        d[np.flatnonzero(out.view(np.uint32) != ref.view(np.uint32))[:5]]
    nan = gm.gm_convert(torch.tensor([np.nan], dtype=torch.float64).cuda()).cpu().numpy()
    assert np.isnan(nan[0])


def test_convert_rejects_bad_arguments(gm):
    lib = gm.load()
    assert lib.gm_convert(2, 4, 1, 1, None) == gm.GM_ERR_ARG
    assert lib.gm_convert(0, -1, None, None, None) == gm.GM_ERR_ARG
    assert lib.gm_convert(0, 3, None, None, None) == gm.GM_ERR_ARG
    assert lib.gm_convert(0, 0, None, None, None) == gm.GM_OK
