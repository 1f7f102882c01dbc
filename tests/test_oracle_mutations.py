"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a scratch copy of the oracle (oracle.c or
net.py, on the CPU), runs the CPU pin tests against that copy in a child
pytest, and expects a test failure.  An unmodified copy must pass the same
run, so a failure is the planted mistake's and not the harness's.  The
mistakes are the ones a restatement of Sec. 2.1-2.2 and of the learned
decimation is most likely to make: a wrong power of U, a dropped cosine
weight, a sign in Eq. 1, the row formula, the 2 pi / P versus pi / P scale,
the Ram-Lak sign, a tap index or normalisation off, the crop bounds, the
shift back, the representative view of a decimated group, and in the
learned decimation a transposed channel matrix, a tap offset, a missing
ReLU, the adjoint's weights and the BF16 significand width.

Two mistakes are deliberately absent: dropping the x or the a2 term of
net.act_rounding_bound leaves a valid (smaller) bound, because
a2 <= sum |W2| (a1 + e1) by the triangle inequality, so no pin can or should
reject it."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = ["test_oracle_bounds.py", "test_oracle_fdk.py", "test_oracle_fdkod.py", "test_oracle_filter.py",
        "test_oracle_taps.py", "test_oracle_net.py", "test_learn.py"]

SHIFT = "lerp_row(Q, off, Nu, (p + (double)w0) + (double)t)"
SHIFT_ROWS = "lerp_row(qb, off, Nu, (p + (double)w0) + (double)t)"

# (name, file under oracle/, text, replacement of every occurrence)
MUTATIONS = [
    ("U^-1 weight for U^-2", "oracle.c", "acc += val / (U * U);", "acc += val / U;"),
    ("no cosine weight", "oracle.c", "q[m] = (double)p[m] * R / sqrt(R * R + a * a + b * b);",
     "q[m] = (double)p[m];"),
    ("no row offset b in the cosine weight", "oracle.c", "sqrt(R * R + a * a + b * b)", "sqrt(R * R + a * a)"),
    ("sign of Eq. 1's numerator", "oracle.c", "double num = y * cb - x * sb;", "double num = x * sb - y * cb;"),
    ("row z U instead of z / U", "oracle.c", "double v = z / U + vc;", "double v = z * U + vc;"),
    ("sign of the magnification's x, y terms", "oracle.c", "return (R + x * cb + y * sb) / R;",
     "return (R - x * cb - y * sb) / R;"),
    ("2 pi / P scale in plain FDK", "oracle.c", "(M_PI / (double)P) * acc", "(2.0 * M_PI / (double)P) * acc"),
    ("Ram-Lak sign", "oracle.c", "return -1.0 / (M_PI * M_PI * dn * dn);", "return 1.0 / (M_PI * M_PI * dn * dn);"),
    ("shift by phi - w0", "oracle.c", SHIFT, "lerp_row(Q, off, Nu, (p - (double)w0) + (double)t)"),
    ("triangle taps normalised by D instead of D^2", "oracle.c",
     "(double)(D - abs(i)) / ((double)D * (double)D)", "(double)(D - abs(i)) / (double)D"),
    ("angular tap index off by one", "oracle.c", "int k = ((j * D + i) % P + P) % P;",
     "int k = ((j * D + i + 1) % P + P) % P;"),
    ("shift back with + w0", "oracle.c", "*t = u - o->phi[(size_t)q * o->P + k] - (double)o->w0[q];",
     "*t = u - o->phi[(size_t)q * o->P + k] + (double)o->w0[q];"),
    ("pi / P instead of pi / P' after decimation", "oracle.c", "return (M_PI / (double)o->Pd) * acc;",
     "return (M_PI / (double)o->P) * acc;"),
    ("hi one column short", "oracle.c", "hi[q * P + k] = (int32_t)floor(umax) + 1;",
     "hi[q * P + k] = (int32_t)floor(umax);"),
    ("a vertex for the square's centre", "oracle.c", "double p = eq1_a(R, xc, yc, cb, sb) + uc;",
     "double p = eq1_a(R, xs[0], ys[0], cb, sb) + uc;"),
    ("representative view jD + 1", "oracle.c", "int k = j * o->D;", "int k = (j * o->D + 1) % o->P;"),
    ("no left margin in w0", "oracle.c", "int32_t w = (int32_t)floor(dmin) - 1;",
     "int32_t w = (int32_t)floor(dmin) + 1;"),
    ("T one column short", "oracle.c", "T[q] = (int32_t)floor(dmax) + 3 - w;", "T[q] = (int32_t)floor(dmax) + 2 - w;"),
    ("squares one voxel short", "oracle.c", "*i1 = (int)((((long)q + 1) * N + m - 1) / m) - 1;",
     "*i1 = (int)((((long)q + 1) * N + m - 1) / m) - 2;"),
    ("shifted rows of the learned path with - w0", "oracle.c", SHIFT_ROWS,
     "lerp_row(qb, off, Nu, (p - (double)w0) + (double)t)"),
    ("adjoint without U^-2", "oracle.c", "double g = scale * e / (U * U);", "double g = scale * e;"),
    ("adjoint's bilinear weights transposed", "oracle.c",
     "{{(1.0 - fr) * (1.0 - fc), (1.0 - fr) * fc}, {fr * (1.0 - fc), fr * fc}}",
     "{{(1.0 - fr) * (1.0 - fc), fr * (1.0 - fc)}, {(1.0 - fr) * fc, fr * fc}}"),
    ("adjoint scale pi / P", "oracle.c", "double scale = M_PI / (double)o.Pd;", "double scale = M_PI / (double)o.P;"),
    ("layer 2 with the channel matrix transposed", "net.py",
     "z2 += np.tensordot(W2[:, :, m], _ahead(a1, m - 2), axes=(1, 0))",
     "z2 += np.tensordot(W2[:, :, m].T, _ahead(a1, m - 2), axes=(1, 0))"),
    ("layer 3 tap offset m - 1", "net.py", "full = sum(np.tensordot(W3[:, m], _ahead(a2, m - 2), axes=(0, 0))",
     "full = sum(np.tensordot(W3[:, m], _ahead(a2, m - 1), axes=(0, 0))"),
    ("no ReLU on layer 2", "net.py", "a2 = rnd(np.maximum(z2, 0.0))", "a2 = rnd(z2)"),
    ("layer-1 gradient with the tap shift flipped", "net.py", "(dz1 * _ahead(x, m - 2)).sum(axis=red)",
     "(dz1 * _ahead(x, -(m - 2))).sum(axis=red)"),
    ("BF16 rounding to 7 significant bits", "net.py", "scale = np.ldexp(1.0, e - 8)",
     "scale = np.ldexp(1.0, e - 7)"),
]


def _replace(text, old, new):
    assert old in text, f"mutation target not found: {old!r}"
    return text.replace(old, new)


def _scratch(base, name, mutation):
    d = os.path.join(base, name)
    os.makedirs(os.path.join(d, "tests"))
    os.makedirs(os.path.join(d, "oracle"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    for f in ["conftest.py"] + PINS:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests"))
    for f in ("__init__.py", "oracle.c", "net.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(d, "oracle"))
    if mutation is not None:
        _, fname, old, new = mutation
        path = os.path.join(d, "oracle", fname)
        text = open(path).read()
        open(path, "w").write(_replace(text, old, new))
    return d


def _env():
    env = dict(os.environ)
    # the scratch directory comes first (it is the working directory and the
    # conftest's root); the repository supplies the input generator and the
    # package's host modules
    env["PYTHONPATH"] = ROOT + (os.pathsep + env["PYTHONPATH"] if env.get("PYTHONPATH") else "")
    env["OMP_NUM_THREADS"] = "2"
    env.pop("PYTEST_ADDOPTS", None)
    return env


def _run_pins(d):
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
           "-p", "no:randomly"] + [os.path.join("tests", f) for f in PINS]
    r = subprocess.run(cmd, cwd=d, env=_env(), capture_output=True, text=True, timeout=600)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    return r.returncode, summary, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.slow
def test_planted_mistakes_fail_the_pins(tmp_path):
    control = _scratch(str(tmp_path), "control", None)
    where = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], cwd=control,
                           env=_env(), capture_output=True, text=True, timeout=120)
    assert where.returncode == 0 and where.stdout.strip().startswith(control), where.stdout + where.stderr
    rc, _, log = _run_pins(control)
    assert rc == 0, "the unmodified copy must pass:\n" + log

    dirs = [_scratch(str(tmp_path), f"m{i:02d}", m) for i, m in enumerate(MUTATIONS)]
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(_run_pins, dirs))
    # caught = a pin failed (not a collection or fixture error, e.g. a copy
    # that does not compile)
    missed = [(m[0], log) for m, (rc, summary, log) in zip(MUTATIONS, results)
              if rc != 1 or " failed" not in summary or " error" in summary]
    assert not missed, "\n\n".join(f"{name}: not caught by a failing pin\n{log}" for name, log in missed)
