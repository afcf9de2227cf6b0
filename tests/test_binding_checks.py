"""The Python binding refuses tensors that would let a C call read or write
past their end, of the wrong type, off the GPU or strided (CPU: a stand-in
with the four attributes the checks read)."""
import pytest

torch = pytest.importorskip("torch")
from paper_2007_12273_gb300 import gm  # noqa: E402


class T:
    """is_cuda, dtype, is_contiguous() and numel() of a device tensor."""

    def __init__(self, n, dtype=torch.float64, cuda=True, contiguous=True):
        self.n, self.dtype, self.is_cuda, self.c = n, dtype, cuda, contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self.c


def test_check_accepts_and_refuses():
    gm._check(T(10), torch.float64, "a", 10)
    gm._check(T(12), torch.float64, "a", 10)
    gm._check(T(5, torch.int32), gm._STATUS, "s", 5)
    with pytest.raises(ValueError, match="required"):
        gm._check(None, torch.float64, "a")
    with pytest.raises(ValueError, match="CUDA"):
        gm._check(T(10, cuda=False), torch.float64, "a")
    with pytest.raises(ValueError, match="must be torch.float64"):
        gm._check(T(10, torch.float32), torch.float64, "a")
    with pytest.raises(ValueError, match="contiguous"):
        gm._check(T(10, contiguous=False), torch.float64, "a")
    with pytest.raises(ValueError, match="at least 11"):
        gm._check(T(10), torch.float64, "a", 11)


def test_mixtures_and_outputs():
    cfg = gm.config(dict(D=3, Kmax=4, shape_order=2, L=1.0))
    C, P = 7, gm.P_of(3)
    good = (T(C, torch.int32), T(C * 4 * P), T(C), T(C))
    gm._check_mixtures(cfg, C, *good)
    with pytest.raises(ValueError, match="params"):
        gm._check_mixtures(cfg, C, good[0], T(C * 4 * P - 1), good[2], good[3])
    with pytest.raises(ValueError, match="K must be torch.int32"):
        gm._check_mixtures(cfg, C, T(C, torch.int64), *good[1:])
    n = 20
    out = dict(x=T(n), v=T(3 * n), alpha=T(n), status=T(C, torch.int32))
    gm._check_recon_out(out, 3, C, n)
    with pytest.raises(ValueError, match="missing 'y'"):
        gm._check_recon_out(out, 3, C, n, two_d=True)
    out["dA"] = T(C - 1)
    with pytest.raises(ValueError, match="dA"):
        gm._check_recon_out(out, 3, C, n)
    out["dA"] = None  # optional
    gm._check_recon_out(out, 3, C, n)
    out["v"] = T(3 * n - 1)
    with pytest.raises(ValueError, match="'v'"):
        gm._check_recon_out(out, 3, C, n)


def test_particles():
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=2, L=1.0))

    class V(T):
        def __init__(self, shape, dtype=torch.float32):
            super().__init__(shape[0] * shape[1], dtype)
            self.shape = shape

    n = 9
    gm._check_particles(cfg, T(4, torch.int64), T(n), V((1, n)), T(n), n)
    gm._check_particles(cfg, T(4, torch.int64), None, V((1, n), torch.float64), T(n), n)
    with pytest.raises(ValueError, match=r"v must be \[D, n\]"):
        gm._check_particles(cfg, T(4, torch.int64), T(n), V((3, n)), T(n), n)
    with pytest.raises(ValueError, match="alpha"):
        gm._check_particles(cfg, T(4, torch.int64), T(n), V((1, n)), T(n - 1), n)
    with pytest.raises(ValueError, match="cell_off"):
        gm._check_particles(cfg, T(4, torch.int32), T(n), V((1, n)), T(n), n)


def test_network_rows():
    import types

    class X(T):
        def __init__(self, shape, dtype=torch.bfloat16):
            super().__init__(shape[0] * shape[1], dtype)
            self.shape = shape

        def dim(self):
            return len(self.shape)

    net = types.SimpleNamespace(F=gm.feat_width(1))
    assert gm.Net._check_rows(net, X((32, 128))) == 32
    with pytest.raises(ValueError, match=r"\[M, 128\]"):
        gm.Net._check_rows(net, X((32, 576)))
    with pytest.raises(ValueError, match="bfloat16"):
        gm.Net._check_rows(net, X((32, 128), torch.float32))
