"""Writes bounds_*.txt: the crop bounds of Sec. 2.1 (Eq. 1 at each square's
four vertex voxel centres) for the 4^s squares of Sec. 2.2, on small
geometries with ragged squares, as computed by the FP64 oracle alone.

    python tests/golden/make_bounds.py

The paper prints no worked example of these numbers; the fixtures freeze
the oracle's values, which tests/test_oracle_bounds.py pins independently
(brute-force projection of every voxel centre of the squares), so a later
change to the oracle's bound arithmetic shows up as a fixture mismatch.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

# (R, N, Nu, P, s): odd N so that 2^s does not divide it; a short source
# distance so that the magnification varies strongly across a square
CASES = [(20.5, 13, 24, 12, 2), (9.25, 10, 27, 8, 1)]


def name(R, N, Nu, P, s):
    return f"bounds_R{R:g}_N{N}_Nu{Nu}_P{P}_s{s}.txt"


def write(R, N, Nu, P, s):
    b = oracle.bounds(R, N, Nu, P, s)
    lines = [f"# crop bounds (Sec. 2.1 Eq. 1 at the vertices; Sec. 2.2 squares), written by make_bounds.py",
             f"# R N Nu P s", f"{R!r} {N} {Nu} {P} {s}",
             "# per square q: w0 T",
             *[f"{int(b['w0'][q])} {int(b['T'][q])}" for q in range(4 ** s)],
             "# per square q, view k: lo hi crop phi (phi as a hexadecimal FP64)",
             *[f"{int(b['lo'][q, k])} {int(b['hi'][q, k])} {int(b['crop'][q, k])} {float(b['phi'][q, k]).hex()}"
               for q in range(4 ** s) for k in range(P)]]
    with open(os.path.join(HERE, name(R, N, Nu, P, s)), "w") as f:
        f.write("\n".join(lines) + "\n")


def read(path):
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    R, N, Nu, P, s = float(rows[0][0]), *map(int, rows[0][1:])
    nsq = 4 ** s
    sq = rows[1:1 + nsq]
    vw = rows[1 + nsq:]
    assert len(vw) == nsq * P
    import numpy as np
    return {"geometry": (R, N, Nu, P, s),
            "w0": np.array([int(r[0]) for r in sq], np.int32),
            "T": np.array([int(r[1]) for r in sq], np.int32),
            "lo": np.array([int(r[0]) for r in vw], np.int32).reshape(nsq, P),
            "hi": np.array([int(r[1]) for r in vw], np.int32).reshape(nsq, P),
            "crop": np.array([int(r[2]) for r in vw], np.int32).reshape(nsq, P),
            "phi": np.array([float.fromhex(r[3]) for r in vw], np.float64).reshape(nsq, P)}


if __name__ == "__main__":
    for c in CASES:
        write(*c)
