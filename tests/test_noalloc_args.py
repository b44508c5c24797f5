"""Argument checks of the direct_noalloc wrapper, on the CPU.

The wrapper must refuse, before the native call, every input the kernel would read or write
out of bounds: a q with the wrong row count, an `out` of the wrong shape, dtype, layout or
device, and tensors on different devices.  CUDA tensors are stood in for by a thin wrapper
that reports a CUDA device; the native library is never reached in these cases.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_0911_4114_gb300.plan import direct_noalloc  # noqa: E402


class FakeCuda:
    """A CPU tensor that presents itself as a CUDA tensor on `device`."""
    is_cuda = True

    def __init__(self, t, device="cuda:0"):
        self.t = t
        self.device = torch.device(device)

    dtype = property(lambda self: self.t.dtype)
    shape = property(lambda self: self.t.shape)

    def dim(self):
        return self.t.dim()

    def is_contiguous(self):
        return self.t.is_contiguous()

    def reshape(self, *a):
        return FakeCuda(self.t.reshape(*a), str(self.device))

    def contiguous(self):
        return self


def _args(ns=5, nt=4, r=2, dtype=torch.complex64):
    s = FakeCuda(torch.zeros(ns, 3, dtype=torch.float64))
    t = FakeCuda(torch.zeros(nt, 3, dtype=torch.float64))
    q = FakeCuda(torch.zeros(ns, r, dtype=dtype))
    return s, t, q


def test_rejects_short_q():
    s, t, _ = _args()
    q = FakeCuda(torch.zeros(4, 2, dtype=torch.complex64))
    with pytest.raises(ValueError, match="rows"):
        direct_noalloc(s, t, q, 1.0)


@pytest.mark.parametrize("bad", ["shape", "dtype", "layout", "device"])
def test_rejects_bad_out(bad):
    s, t, q = _args()
    if bad == "shape":
        out = FakeCuda(torch.zeros(3, 2, dtype=torch.complex64))
    elif bad == "dtype":
        out = FakeCuda(torch.zeros(4, 2, dtype=torch.complex128))
    elif bad == "layout":
        out = FakeCuda(torch.zeros(2, 4, dtype=torch.complex64).t())
    else:
        out = FakeCuda(torch.zeros(4, 2, dtype=torch.complex64), "cuda:1")
    with pytest.raises(ValueError, match="out must be"):
        direct_noalloc(s, t, q, 1.0, out=out)


def test_rejects_mixed_devices():
    s, t, q = _args()
    t = FakeCuda(t.t, "cuda:1")
    with pytest.raises(ValueError, match="one device"):
        direct_noalloc(s, t, q, 1.0)


def test_rejects_bad_points():
    _, t, q = _args()
    s = FakeCuda(torch.zeros(5, 2, dtype=torch.float64))
    with pytest.raises(ValueError, match="sources"):
        direct_noalloc(s, t, q, 1.0)
