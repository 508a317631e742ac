"""The C ABI library loads and exports every function the headers under include/
declare (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ostrich_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2609_08800_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    names = _declared()
    assert "ostrich_step" in names and "ostrich_adjoint" in names and "ostrich_probe_ffma" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_refuses_host_and_strided_arrays():
    """The library reads packed [rows, ld] device arrays; a strided view or a host
    tensor is refused instead of being misread."""
    import pytest
    from paper_2609_08800_gb300.ostrich import _ptr

    class Fake:
        def __init__(self, cuda, contig):
            self.is_cuda, self._c, self.shape = cuda, contig, (4, 3)

        def is_contiguous(self):
            return self._c

        def stride(self):
            return (1, 4)

        def data_ptr(self):
            return 4096

    assert _ptr(None) is None
    assert _ptr(Fake(True, True)).value == 4096
    with pytest.raises(ValueError):
        _ptr(Fake(False, True))
    with pytest.raises(ValueError):
        _ptr(Fake(True, False))
