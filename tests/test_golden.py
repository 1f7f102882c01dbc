"""Stored crop bounds (tests/golden/bounds_*.txt, written by
tests/golden/make_bounds.py from the oracle alone).

The paper prints no worked example, so the fixtures are the oracle's own
values on small geometries with ragged squares.  Here they are checked
against a brute-force projection of every voxel centre of each square (ray
and detector-plane algebra, not Eq. 1), and the oracle must still reproduce
them bit for bit; the CUDA library is compared with the same files in
test_gpu_parity.py."""
import glob
import os

import numpy as np
import pytest

from test_oracle_bounds import _project_u, _squares

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = sorted(glob.glob(os.path.join(HERE, "golden", "bounds_*.txt")))


def _read(path):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_bounds", os.path.join(HERE, "golden", "make_bounds.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.read(path)


def test_fixtures_present():
    assert len(FILES) >= 2


@pytest.mark.parametrize("path", FILES, ids=os.path.basename)
def test_oracle_reproduces_the_stored_bounds(oracle_mod, path):
    g = _read(path)
    b = oracle_mod.bounds(*g["geometry"])
    for key in ("lo", "hi", "crop", "w0", "T"):
        assert np.array_equal(b[key], g[key]), key
    assert np.array_equal(b["phi"].view(np.int64), g["phi"].view(np.int64))


@pytest.mark.parametrize("path", FILES, ids=os.path.basename)
def test_stored_bounds_match_brute_force(path):
    g = _read(path)
    R, N, Nu, P, s = g["geometry"]
    groups = _squares(N, s)
    m = 2 ** s
    for qy in range(m):
        for qx in range(m):
            q = qy * m + qx
            xs = groups[qx] - (N - 1) / 2
            ys = groups[qy] - (N - 1) / 2
            X, Y = np.meshgrid(xs, ys)
            u = _project_u(R, Nu, P, X, Y)                       # [P][voxels]
            umin, umax = u.min(axis=1), u.max(axis=1)
            assert np.all(np.abs(umin - np.round(umin)) > 1e-9) and np.all(np.abs(umax - np.round(umax)) > 1e-9)
            assert np.array_equal(g["lo"][q], np.floor(umin).astype(np.int32))
            assert np.array_equal(g["hi"][q], np.floor(umax).astype(np.int32) + 1)
            # the shift centre is the projection of the square's centre
            xc, yc = 0.5 * (xs[0] + xs[-1]), 0.5 * (ys[0] + ys[-1])
            phi = _project_u(R, Nu, P, np.array([xc]), np.array([yc]))[:, 0]
            np.testing.assert_allclose(g["phi"][q], phi, rtol=0, atol=1e-9)
            w0 = int(np.floor((umin - g["phi"][q]).min())) - 1
            assert g["w0"][q] == w0
            assert g["T"][q] == int(np.floor((umax - g["phi"][q]).max())) + 3 - w0
            assert np.array_equal(g["crop"][q], np.floor(g["phi"][q] + w0).astype(np.int32))
