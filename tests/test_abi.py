"""The C-ABI library builds for sm_103a, loads and exports every entry point
include/fdkod.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_07515_gb300 import build, fdkod
    build.build()
    return fdkod.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "fdkod.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:fdkod|fdk)_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"fdkod_plan", "fdkod_filter", "fdkod_backproject", "fdk_backproject_plain"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_1708_07515_gb300 import fdkod as F
    out = ctypes.c_void_p()
    assert lib.fdkod_plan(None, 1, 1, 0, ctypes.byref(out)) == -1
    bad = [
        (F.Geometry(64.0, 0, 16, 16, 8), 1, 1, 0, -1),     # N = 0 (empty volume)
        (F.Geometry(64.0, 16, 16, 16, 0), 1, 1, 0, -1),    # no views
        (F.Geometry(-1.0, 16, 16, 16, 8), 1, 1, 0, -1),    # R <= 0
        (F.Geometry(64.0, 16, 16, 16, 8), 1, 1, 7, -1),    # unknown storage type
        (F.Geometry(64.0, 16, 16, 16, 8), 1, 3, 0, -2),    # D does not divide P
        (F.Geometry(64.0, 16, 16, 16, 8), 5, 1, 0, -2),    # 2^s > N
        (F.Geometry(10.0, 16, 16, 16, 8), 1, 1, 0, -2),    # source inside the volume
        (F.Geometry(64.0, 16, 16, 16, 8), -1, 1, 0, -2),   # negative s
    ]
    for g, s, D, qt, want in bad:
        assert lib.fdkod_plan(ctypes.byref(g), s, D, qt, ctypes.byref(out)) == want, (g.N, s, D, qt)
        assert out.value is None
    g = F.Geometry(64.0, 16, 16, 16, 8)
    assert lib.fdkod_plan_ex(ctypes.byref(g), 1, 1, 0, 4, ctypes.byref(out)) == -1   # unknown flag
    g256 = F.Geometry(1024.0, 256, 256, 256, 512)
    assert lib.fdkod_plan(ctypes.byref(g256), 1, 256, 0, ctypes.byref(out)) == -2    # D above 128
    assert lib.fdkod_set_decimation_taps(None, None, 4) == -1
    assert lib.fdkod_get_decimation_taps(None, None, 0) == -1
    assert lib.fdkod_sinc_taps(0, 2, None) == -1
    assert lib.fdkod_slab_rows(None, 0, 1, None, None) == -1
    assert lib.fdkod_filter_rows(None, None, 0, 1, None, 0) == -1
    assert lib.fdkod_backproject_slab(None, None, 0, 1, None, 0, 1, None, 0) == -1
    assert lib.fdkod_set_decimation_net(None, None, 0) == -1
    assert lib.fdkod_get_decimation_net(None, None, 0) == -1
    assert lib.fdkod_net_adjoint(None, None, None, 0, None, None, 0) == -1
    assert lib.fdkod_net_backward(None, None, None, None, 0, 1, None, 0) == -1
    assert lib.fdkod_batch_create(None, None, None, 0, None) == -1
    assert lib.fdkod_set_tile(None, 0) == -1
    assert lib.fdkod_get_tile(None, None, None) == -1
    assert lib.fdkod_batch_backproject(None, 0) == -1
    assert lib.fdkod_reconstruct(None, None, None, 0) == -1
    assert lib.fdkod_set_test_fault(None, 0, 0) == -1
    lib.fdkod_batch_destroy(None)
    for rc in (0, -1, -2, -3, -4, -5, -6, 99):
        assert lib.fdkod_strerror(rc)
    assert lib.fdkod_filter(None, None, None, 0) == -1
    assert lib.fdkod_backproject(None, None, None, 0) == -1
    assert lib.fdk_backproject_plain(None, None, None, 0) == -1
    assert lib.fdkod_get_info(None, None) == -1
    lib.fdkod_destroy(None)


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_1708_07515_gb300 import fdkod as F
    monkeypatch.setattr(F, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(F, "_lib", None)
    with pytest.raises(RuntimeError):
        F.load()


@pytest.mark.parametrize("D,H", [(1, 1), (1, 2), (2, 2), (3, 1), (4, 2), (16, 2), (128, 2)])
def test_library_sinc_taps_match_the_oracle(lib, oracle_mod, D, H):
    """Host-only entry (no device work): the library's windowed sinc and the
    oracle's, written separately from the same definition."""
    from paper_1708_07515_gb300 import fdkod as F
    import numpy as np
    got = F.fdkod_sinc_taps(D, H)
    np.testing.assert_allclose(got, oracle_mod.sinc_taps(D, H), rtol=0, atol=1e-15)
    assert lib.fdkod_sinc_taps(D, 3, None) == -1


def test_binding_signatures_match_the_header():
    """The binding declares every prototype of include/fdkod.h, and nothing
    else, with the same number of parameters."""
    import re as _re
    src = open(os.path.join(ROOT, "include", "fdkod.h")).read()
    src = _re.sub(r"/\*.*?\*/", "", src, flags=_re.S)
    protos = {}
    for m in _re.finditer(r"\b((?:fdkod|fdk)_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src, flags=_re.S):
        args = m.group(2).strip()
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    binding = open(os.path.join(ROOT, "paper_1708_07515_gb300", "fdkod.py")).read()
    table = binding[binding.index("sig = {"):binding.index("for name, (res, args) in sig.items()")]
    bound = {}
    for m in _re.finditer(r'"((?:fdkod|fdk)_[a-z_]+)":\s*\(([^\[]*)\[(.*?)\]\)', table, flags=_re.S):
        inner = m.group(3)
        depth, n = 0, 0
        for ch in inner:
            depth += ch in "(["
            depth -= ch in ")]"
            if ch == "," and depth == 0:
                n += 1
        bound[m.group(1)] = 0 if not inner.strip() else n + 1
    assert len(protos) >= 30
    assert set(bound) == set(protos), set(bound) ^ set(protos)
    for name, n in bound.items():
        assert protos[name] == n, (name, protos[name], n)


class _FakeDev:
    """Stands in for a CUDA tensor (attributes only; nothing is launched)."""

    def __init__(self, shape, dtype, contiguous=True):
        self.is_cuda, self.shape, self.dtype, self._c = True, tuple(shape), dtype, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        n = 1
        for e in self.shape:
            n *= int(e)
        return n


def test_binding_checks_what_the_bare_pointers_cannot():
    """The Plan methods check shape, dtype and layout before a pointer
    reaches the library, so a wrongly sized tensor is a ValueError, not an
    out-of-bounds access on the device."""
    torch = pytest.importorskip("torch")
    from paper_1708_07515_gb300 import fdkod as F
    ok = _FakeDev((4, 5, 6), torch.float32)
    assert F._expect(ok, (4, 5, 6), torch.float32, "x") is ok
    assert F._expect(ok, (4, None, 6), torch.float32, "x") is ok
    assert F._expect(ok, 120, torch.float32, "x", at_least=True) is ok
    for bad, shape, dtype in [(_FakeDev((4, 5, 6), torch.float64), (4, 5, 6), torch.float32),
                              (_FakeDev((4, 5, 7), torch.float32), (4, 5, 6), torch.float32),
                              (_FakeDev((4, 30), torch.float32), (4, 5, 6), torch.float32),
                              (_FakeDev((4, 5, 6), torch.float32, contiguous=False), (4, 5, 6), torch.float32),
                              (torch.zeros((4, 5, 6)), (4, 5, 6), torch.float32)]:
        with pytest.raises(ValueError):
            F._expect(bad, shape, dtype, "x")
    with pytest.raises(ValueError):
        F._expect(ok, 121, torch.float32, "x", at_least=True)
    # the allocation-free entry point knows its shapes from the geometry
    N, P = 8, 6
    with pytest.raises(ValueError):
        F.fdkod_backproject_noalloc(32.0, N, N, N, P, 1, 2, _FakeDev((P, N, N + 1), torch.float32),
                                    _FakeDev((N, N, N), torch.float32))
    with pytest.raises(ValueError):
        F.fdkod_backproject_noalloc(32.0, N, N, N, P, 1, 2, _FakeDev((P, N, N), torch.float32),
                                    _FakeDev((N, N, N), torch.float16))
