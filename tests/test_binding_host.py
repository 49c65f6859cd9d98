"""The binding's checks of device arrays, on the host: a tensor that is not on the GPU, of the wrong element type,
not contiguous or of the wrong size is refused before its address reaches the library (which would read past a
smaller buffer or through a host pointer), while sizes the library itself refuses still reach it and come back as
its VF_ESIZE."""
import pytest

from paper_2204_02107_gb300 import native

torch = pytest.importorskip("torch")


class FakeCudaTensor:
    """Stands in for a CUDA tensor: only the attributes the binding reads."""

    def __init__(self, n, dtype="float64", contiguous=True):
        self._n, self.dtype, self._contiguous = n, getattr(torch, dtype), contiguous
        self.is_cuda = True

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        return 4096

    def element_size(self):
        return torch.empty(0, dtype=self.dtype).element_size()


FakeCudaTensor.__module__ = "torch.fake"       # the binding recognises tensors by their module


class FakeLib:
    def __init__(self):
        self.calls = []

    def vf_status_string(self, code):
        return b"VF_ESIZE" if code == native.VF_ESIZE else b"VF_OTHER"

    def vf_poisson_noalloc_max_cells(self, precision):
        return 4194304 if precision == native.VF_FP64 else 8388608

    def vf_poisson_solve_noalloc(self, *args):
        self.calls.append(args[:3])
        nx, ny, nz = args[:3]
        return native.VF_ESIZE if nx * ny * nz > 4194304 or nx // 2 + 1 > 1024 else native.VF_OK


@pytest.fixture
def fake_lib(monkeypatch):
    fl = FakeLib()
    monkeypatch.setattr(native, "lib", lambda: fl)
    return fl


def test_device_tensor_checks():
    ok = FakeCudaTensor(10)
    assert native._device_tensor(ok, ("float64",), 10, "x") is ok
    cases = [(torch.zeros(10, dtype=torch.float64), TypeError),          # host tensor
             (FakeCudaTensor(10, "float32"), TypeError),                   # wrong element type
             (FakeCudaTensor(10, contiguous=False), ValueError),
             (FakeCudaTensor(9), ValueError)]
    for x, err in cases:
        with pytest.raises(err):
            native._device_tensor(x, ("float64",), 10, "x")
    with pytest.raises(TypeError):                 # a float mask where bytes are expected
        native._pointer(FakeCudaTensor(10, "float32"), "uint8", 10)
    ptr, mem, _ = native._pointer(FakeCudaTensor(10, "uint8"), "uint8", 10)
    assert mem == native.VF_DEVICE and ptr.value == 4096


def test_noalloc_checks_arrays_only_for_sizes_it_accepts(fake_lib):
    f = FakeCudaTensor(8)
    # sizes the call refuses (over the FP64 cell limit; an x transform longer than 1024) reach it with any array
    for shape in ((512, 128, 128), (2048, 8, 8)):
        with pytest.raises(native.VentflowError) as e:
            native.poisson_solve_noalloc(*shape, 1.0, 1.0, 1.0, f, f)
        assert e.value.code == native.VF_ESIZE
    assert fake_lib.calls == [(512, 128, 128), (2048, 8, 8)]
    # accepted sizes: the arrays must hold one value per cell, p in f's precision
    with pytest.raises(ValueError):
        native.poisson_solve_noalloc(72, 36, 20, 1.0, 1.0, 1.0, f, f)
    n = 72 * 36 * 20
    with pytest.raises(TypeError):
        native.poisson_solve_noalloc(72, 36, 20, 1.0, 1.0, 1.0, FakeCudaTensor(n), FakeCudaTensor(n, "float32"))
    with pytest.raises(TypeError):
        native.poisson_solve_noalloc(72, 36, 20, 1.0, 1.0, 1.0, torch.zeros(n, dtype=torch.float64),
                                     torch.zeros(n, dtype=torch.float64))
    assert len(fake_lib.calls) == 2
    native.poisson_solve_noalloc(72, 36, 20, 1.0, 1.0, 1.0, FakeCudaTensor(n), FakeCudaTensor(n))
    assert fake_lib.calls[-1] == (72, 36, 20)


def test_batch_add_refuses_mixed_host_and_device_inputs(monkeypatch):
    calls = []
    b = native.Batch.__new__(native.Batch)            # no device batch: the check comes before the library call
    b._h, b._desc = None, {}
    monkeypatch.setattr(native, "lib", lambda: type("L", (), {"vf_batch_add": lambda *a: calls.append(a)})())
    desc = native.VfGridDesc()
    desc.nx, desc.ny, desc.nz = 8, 8, 8
    n = 512
    host = __import__("numpy").ones(n, dtype="uint8")
    with pytest.raises(ValueError):
        b.add(desc, host, host, (1.0, 0.0, 0.0), 0.0, 10, room=host, c0=FakeCudaTensor(n))
    with pytest.raises(TypeError):                 # a device c0 must be float64 or float32
        b.add(desc, FakeCudaTensor(n, "uint8"), None, (1.0, 0.0, 0.0), 0.0, 10, c0=FakeCudaTensor(n, "int32"))
    assert calls == []


def test_batch_add_passes_the_element_type_of_c0(monkeypatch):
    """a float32 c0 (host or device) reaches the library as float32 (c0_is_fp64 = 0), anything else as float64"""
    np = __import__("numpy")
    calls = []
    b = native.Batch.__new__(native.Batch)
    b._h, b._desc = None, {}
    monkeypatch.setattr(native, "lib", lambda: type("L", (), {"vf_batch_add": lambda *a: calls.append(a) or 0})())
    desc = native.VfGridDesc()
    desc.nx, desc.ny, desc.nz = 8, 8, 8
    n = 512
    host = np.ones(n, dtype="uint8")
    b.add(desc, host, host, (1.0, 0.0, 0.0), 0.0, 10, room=host, c0=np.ones(n, dtype=np.float32))
    b.add(desc, host, host, (1.0, 0.0, 0.0), 0.0, 10, room=host, c0=np.ones(n))
    dev = FakeCudaTensor(n, "uint8")
    b.add(desc, dev, None, (1.0, 0.0, 0.0), 0.0, 10, c0=FakeCudaTensor(n, "float32"))
    b.add(desc, dev, None, (1.0, 0.0, 0.0), 0.0, 10, c0=FakeCudaTensor(n, "float64"))
    assert [c[9] for c in calls] == [0, 1, 0, 1]   # the c0_is_fp64 argument (after the bound stand-in)
