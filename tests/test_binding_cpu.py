"""CPU checks of the binding's argument checks on device tensors: the C ABI
takes bare pointers, so a tensor of the wrong size, element type or device
must be refused in Python before any library call (a wrong size would let
a kernel read or write out of bounds)."""
import numpy as np
import pytest

from paper_1705_11092_gb300 import clbm


class FakeDevice:
    def __init__(self, index):
        self.index = index


class FakeCudaTensor:
    """Enough of a torch CUDA tensor for the binding's checks."""

    def __init__(self, n, dtype="float64", device=0, contiguous=True):
        import torch
        self._n = n
        self.dtype = torch.float64 if dtype == "float64" else torch.uint8
        self.is_cuda = True
        self.device = FakeDevice(device)
        self._contiguous = contiguous

    def element_size(self):
        return 8 if self.dtype.is_floating_point else 1

    def is_contiguous(self):
        return self._contiguous

    def numel(self):
        return self._n

    def data_ptr(self):
        return 0x1000


class RecordingLib:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append(name)
            return 0
        return fn


@pytest.fixture
def fake(monkeypatch):
    lib = RecordingLib()
    monkeypatch.setattr(clbm, "load", lambda: lib)
    monkeypatch.setattr(clbm, "_current_device", lambda: 0)
    return lib


NX, NY = 20, 10


def _noalloc(f, solid, out):
    clbm.clbm_reduce_noalloc(f, NX, NY, 0.0, 0.0, solid, out, None)


def test_reduce_noalloc_accepts_right_sizes(fake):
    _noalloc(FakeCudaTensor(9 * NX * NY), FakeCudaTensor(NX * NY, "uint8"), FakeCudaTensor(4))
    assert fake.calls == ["clbm_reduce_noalloc"]


@pytest.mark.parametrize("f,solid,out", [
    (9 * NX * NY - 1, NX * NY, 4),        # f too small
    (9 * NX * NY + 9, NX * NY, 4),        # f of another lattice
    (9 * NX * NY, NX * NY - 1, 4),        # solid too small
    (9 * NX * NY, NX * NY, 3),            # out too small
])
def test_reduce_noalloc_rejects_wrong_sizes_before_the_library(fake, f, solid, out):
    with pytest.raises(ValueError):
        _noalloc(FakeCudaTensor(f), FakeCudaTensor(solid, "uint8"), FakeCudaTensor(out))
    assert fake.calls == []


def test_reduce_noalloc_rejects_other_devices_and_types(fake):
    with pytest.raises(ValueError):
        _noalloc(FakeCudaTensor(9 * NX * NY, device=1), None, FakeCudaTensor(4))
    with pytest.raises(ValueError):
        _noalloc(FakeCudaTensor(9 * NX * NY), FakeCudaTensor(NX * NY), FakeCudaTensor(4))   # solid not uint8
    with pytest.raises(ValueError):
        _noalloc(FakeCudaTensor(9 * NX * NY, contiguous=False), None, FakeCudaTensor(4))
    assert fake.calls == []


def test_device_field_calls_check_the_lattice_size(fake, monkeypatch):
    monkeypatch.setattr(clbm, "clbm_get_size", lambda h: (NX, NY))
    clbm.clbm_moments_dev(None, FakeCudaTensor(NX * NY), None, None)
    clbm.clbm_init_dev(None, None, FakeCudaTensor(NX * NY), FakeCudaTensor(NX * NY))
    assert fake.calls == ["clbm_moments_dev", "clbm_init_dev"]
    for bad in (NX * NY - 1, NX * NY + 1):
        with pytest.raises(ValueError):
            clbm.clbm_moments_dev(None, FakeCudaTensor(bad))
        with pytest.raises(ValueError):
            clbm.clbm_init_dev(None, FakeCudaTensor(bad))
    assert fake.calls == ["clbm_moments_dev", "clbm_init_dev"]


def test_host_population_calls_check_the_lattice_size(fake, monkeypatch):
    monkeypatch.setattr(clbm, "clbm_get_size", lambda h: (NX, NY))
    with pytest.raises(ValueError):
        clbm.clbm_set_populations(None, np.zeros((9, NY, NX - 1)))
    with pytest.raises(ValueError):
        clbm.clbm_get_populations(None, np.zeros((9, NY + 1, NX)))
    assert fake.calls == []
    clbm.clbm_get_populations(None, np.zeros((9, NY, NX)), pre_collision=True)
    assert fake.calls == ["clbm_get_populations"]
