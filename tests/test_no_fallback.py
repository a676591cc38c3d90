"""The product path has no CPU fallback: without the compiled library the
binding refuses to load, and without a CUDA device the library's set-up fails
with an error status instead of computing anything on the host."""
import pytest

import gemslr_inputs as gi


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2205_03224_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libgemslr.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_setup_without_a_device_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2205_03224_gb300 import Gemslr, _lib, build, partition_geometric
    build.build()
    A, xyz = gi.grid_operator((8, 7))
    part = partition_geometric(A, xyz, 2, 2)            # host logic: allowed without a device
    for alloc in ("torch", None):
        with pytest.raises(_lib.GemslrError):
            Gemslr(A, part, ilu="ilu0", rank=2, allocator=alloc)
