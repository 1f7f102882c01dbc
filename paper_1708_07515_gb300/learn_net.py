"""Training of the learned angular decimation (the residual conv net of
fdkod_set_decimation_net) with the library's own kernels.

Sec. 2.1 leaves the angular low-pass open and says its implementation sets
the quality; full FDK (D = 1, the same decomposition without decimation)
is the reconstruction FDK-OD approximates, so it is the target.  Per step,
for one training scan (filtered projections Q on the device) and a batch of
slices:

  1. S' = the decomposition with the current weights (the tensor-core
     inference kernel: BF16 weights and layer inputs, FP32 accumulation);
  2. f = the FDK-OD backprojection of S';
  3. per slice z, fdkod_net_adjoint turns e = f[z] - f_FDK[z] into dS, the
     gradient of (1/2) sum e^2 with respect to S';
  4. fdkod_net_backward turns dS into the weight gradient (FP32 master
     weights, forward recomputed in FP32: the BF16 rounding of inference is
     passed straight through);
  5. Adam on the 1440 master weights (host).

The loss is sum e^2 / sum f_FDK^2 over the step's slices.  Layer 3 starts
at zero, so training starts from the plain low-pass.  The plain low-pass is
the triangle, or (--base learned) the linear taps of support 2D fitted to
full FDK on the same training scans (learn.py): the net then learns a
residual on top of the best linear filter, and starts exactly at it.

    python -m paper_1708_07515_gb300.learn_net --N 512 --P 720 --s 3 --D 4

prints the loss curve, the held-out rel-RMSE against full FDK of the
triangle, the windowed sinc and the net, and writes the weights (--out).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

NET_SIZE = 1440


def init_weights(seed: int) -> np.ndarray:
    """He-scaled layers 1 and 2, layer 3 zero (the plain low-pass)."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal(80) * np.sqrt(2.0 / 5.0)
    w2 = rng.standard_normal(1280) * np.sqrt(2.0 / 80.0)
    return np.concatenate([w1, w2, np.zeros(80)]).astype(np.float32)


def linear_config(g: dict, seed: int, scale: float = 0.05) -> np.ndarray:
    """Weights under which the net adds the linear FIR sum_o g[o] x[jD + o]
    (|o| <= 6) to the plain low-pass: channel pairs carry relu(+x) and
    relu(-x) shifted by -4, 0 and +4 views through layers 1 and 2 (relu(u)
    - relu(-u) = u), and layer 3 reads their differences at offsets -6..-3,
    -2..2 and 3..6.  The other 10 channels of layers 1 and 2 get small
    random weights (their layer-3 weights start at zero)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((16, 5)) * scale
    W2 = rng.standard_normal((16, 16, 5)) * scale
    W3 = np.zeros((16, 5))
    W1[:6] = 0.0
    W2[:6] = 0.0
    for p, (shift, offs) in enumerate([(-4, range(-6, -2)), (0, range(-2, 3)), (4, range(3, 7))]):
        cp, cn = 2 * p, 2 * p + 1
        o1 = shift // 2                      # split the shift over layers 1 and 2
        o2 = shift - o1
        W1[cp, o1 + 2], W1[cn, o1 + 2] = 1.0, -1.0
        W2[cp, cp, o2 + 2], W2[cp, cn, o2 + 2] = 1.0, -1.0
        W2[cn, cn, o2 + 2], W2[cn, cp, o2 + 2] = 1.0, -1.0
        for o in offs:
            m = o - shift + 2
            W3[cp, m], W3[cn, m] = g.get(o, 0.0), -g.get(o, 0.0)
    return np.concatenate([W1.reshape(-1), W2.reshape(-1), W3.reshape(-1)]).astype(np.float32)


def linear_fit(R: float, N: int, P: int, s: int, D: int, projs, zs, half: int = 6) -> dict:
    """The symmetric FIR correction g[o] = g[-o], |o| <= half, that, added to
    the plain triangle (whose support |i| < D may reach past it), brings
    FDK-OD closest to full FDK on the training scans, with zero gain at zero
    frequency (the total keeps unit gain).  With B_i the reconstruction from
    the unit tap pair at +-i (library kernels, learn.normal_equations):
    minimise |sum_i (tri_i + g_i) B_i - f_FDK|^2 subject to c . g = 0,
    c = (1, 2, 2, ...), a KKT system of half + 2 unknowns.  Returns
    {offset: g}."""
    from . import learn
    from .fdkod import Plan
    n = half + 1
    H = 2 if max(n, D) > D else 1            # tap blocks: cover |i| <= half and the triangle
    if max(n, D) > 2 * D:
        raise ValueError("the fit's plan takes at most 2 D taps")
    m = H * D
    G = np.zeros((m, m))
    b = np.zeros(m)
    with Plan(R, N, N, N, P, s, D) as pt, Plan(R, N, N, N, P, s, 1) as pf:
        for proj in projs:
            Q = pt.filter(proj)
            gg, bb, _, _ = learn.normal_equations(pt, pf, Q, m, zs)
            G += gg
            b += bb
    tri = np.maximum(D - np.arange(m), 0) / float(D * D)
    g = solve_correction(G, b, tri, n)
    return {o: float(g[abs(o)]) for o in range(-half, half + 1)}


def solve_correction(G: np.ndarray, b: np.ndarray, base: np.ndarray, n: int) -> np.ndarray:
    """argmin over g (n taps g[|i|]) of 1/2 (base + g)^T G (base + g) - b^T g
    subject to g_0 + 2 sum_{i>0} g_i = 0, with G, b over the first
    len(base) taps (g zero past n): the KKT system of half + 2 unknowns."""
    from . import learn
    c = learn.constraint(n)
    K = np.zeros((n + 1, n + 1))
    K[:n, :n] = G[:n, :n]
    K[:n, n] = c
    K[n, :n] = c
    rhs = np.concatenate([b[:n] - G[:n] @ base, [0.0]])
    return np.linalg.solve(K, rhs)[:n]


class Adam:
    def __init__(self, n: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, w: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return (w - self.lr * mh / (np.sqrt(vh) + self.eps)).astype(np.float32)


def merge_rows(ranges):
    """Union of half-open row intervals as disjoint intervals."""
    out = []
    for lo, hi in sorted(ranges):
        if out and lo <= out[-1][1]:
            out[-1][1] = max(out[-1][1], hi)
        else:
            out.append([lo, hi])
    return [tuple(r) for r in out]


class Trainer:
    """Holds one plan (R, N, P, s, D), the training scans' Q and FDK volumes."""

    def __init__(self, R: float, N: int, P: int, s: int, D: int, taps="triangle"):
        import torch

        from .fdkod import Plan
        self.torch = torch
        self.N, self.P, self.D = N, P, D
        self.plan = Plan(R, N, N, N, P, s, D, taps=taps)
        self.ref_plan = Plan(R, N, N, N, P, s, 1)
        info = self.plan.info
        self.dS = torch.zeros((info["n_squares"], info["Pd"], N, info["T_stride"]), device="cuda")
        self.dW = torch.zeros(NET_SIZE, device="cuda")
        self.err = torch.zeros(1, device="cuda")
        self.wdev = torch.zeros(NET_SIZE, device="cuda")
        self.scans = []

    def close(self):
        self.plan.close()
        self.ref_plan.close()

    def add_scan(self, proj):
        """proj: unfiltered projections [P][N][N] (torch CUDA float32)."""
        Q = self.plan.filter(proj)
        ref = self.ref_plan.backproject(Q)
        self.scans.append((Q, ref))

    def loss_and_grad(self, w: np.ndarray, scan: int, zs) -> tuple[float, np.ndarray]:
        torch = self.torch
        Q, ref = self.scans[scan]
        self.plan.set_net(w)
        S = self.plan.decompose(Q)
        vol = self.plan.backproject_decomposed(S)
        self.dS.zero_()
        self.dW.zero_()
        self.err.zero_()
        for z in zs:
            self.plan.net_adjoint(vol[z], ref[z], int(z), self.dS, self.err)
        rows = merge_rows([(v0, v0 + n) for v0, n in (self.plan.slab_rows(int(z), 1) for z in zs)])
        self.wdev.copy_(torch.from_numpy(w))
        for lo, hi in rows:
            self.plan.net_backward(Q, self.wdev, self.dS, lo, hi, self.dW)
        den = float(sum(torch.sum(ref[z].double() ** 2).item() for z in zs))
        loss = self.err.item() / den
        return loss, self.dW.cpu().numpy().astype(np.float64) * (2.0 / den)

    def rel_rmse(self, w, scans, zs) -> float:
        """rel-RMSE against full FDK on the given scans and slices (w None:
        the plain low-pass)."""
        torch = self.torch
        self.plan.set_net(w)
        num = den = 0.0
        for Q, ref in scans:
            vol = self.plan.backproject(Q)
            for z in zs:
                num += float(torch.sum((vol[z].double() - ref[z].double()) ** 2).item())
                den += float(torch.sum(ref[z].double() ** 2).item())
        self.plan.set_net(None)
        return (num / den) ** 0.5


def train(tr: Trainer, steps: int, lr: float, slices: int, seed: int, w0=None, log_every: int = 10,
          val_slices=None):
    """Adam with a linear warm-up (a tenth of the steps) and a cosine-decayed
    step size.  The curve holds (step, loss of
    that step's slices) and, with val_slices, the rel-RMSE on those fixed
    slices of every training scan (the step's own loss depends on which
    slices it drew)."""
    rng = np.random.default_rng(seed)
    w = init_weights(seed) if w0 is None else np.asarray(w0, np.float32)
    opt = Adam(NET_SIZE, lr)
    N = tr.N
    curve = []
    warm = max(1, steps // 10)
    for it in range(steps):
        opt.lr = lr * min(1.0, (it + 1) / warm) * 0.5 * (1.0 + np.cos(np.pi * it / steps))
        scan = it % len(tr.scans)
        zs = rng.integers(N // 10, N - N // 10, size=slices)
        loss, g = tr.loss_and_grad(w, scan, zs)
        w = opt.step(w, g)
        if it % log_every == 0 or it == steps - 1:
            entry = [it, loss]
            if val_slices is not None:
                entry.append(tr.rel_rmse(w, tr.scans, val_slices))
            curve.append(tuple(entry))
    return w, curve


def main(argv=None):
    import torch

    import phantom
    from .fdkod import fdkod_sinc_taps

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--P", type=int, default=720)
    ap.add_argument("--s", type=int, default=3)
    ap.add_argument("--D", type=int, default=4)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--slices", type=int, default=4, help="slices per step")
    ap.add_argument("--train", type=int, default=4, help="training scans (seeds 8000..)")
    ap.add_argument("--test", type=int, default=2, help="held-out scans (seeds 9000..)")
    ap.add_argument("--ellipsoids", type=int, default=40)
    ap.add_argument("--eval-slices", type=int, default=16)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=None, help="write the trained weights here (.npy)")
    ap.add_argument("--log-every", type=int, default=25)
    ap.add_argument("--linear", action="store_true", help="also fit the linear learned FIR (learn.py)")
    ap.add_argument("--init", choices=["linear", "random"], default="linear",
                    help="start at the best linear FIR within the net's reach (13 taps) or at random layers 1-2 "
                         "with a zero layer 3")
    ap.add_argument("--base", choices=["triangle", "learned"], default="triangle",
                    help="plain low-pass under the net: the triangle, or the learned linear taps of support 2D "
                         "(fitted on the training scans; written beside --out as <out>_taps.npy)")
    args = ap.parse_args(argv)
    N, P, s, D = args.N, args.P, args.s, args.D
    R = 4.0 * N
    torch.cuda.set_device(0)

    def scan(seed):
        return phantom.project_gpu(phantom.make_phantom(seed, N, args.ellipsoids), R, N, N, P)

    zs = np.linspace(N // 8, N - 1 - N // 8, args.eval_slices).round().astype(int)
    projs = [scan(8000 + i) for i in range(args.train)]
    base = None
    if args.base == "learned":
        # the best linear taps of support 2D: the net's residual starts there
        from . import learn
        base = learn.learn(R, N, P, s, D, 2, projs, zs)
    tr = Trainer(R, N, P, s, D, taps="triangle" if base is None else base)
    try:
        for p in projs:
            tr.add_scan(p)
        t0 = time.time()
        w0 = None
        if args.init == "linear":
            # the 13-tap linear correction of the base within the net's reach
            # (zero on top of the learned taps, which are already the
            # optimum of a wider support)
            g = linear_fit(R, N, P, s, D, projs, zs) if base is None else {}
            w0 = linear_config(g, args.seed)
        w, curve = train(tr, args.steps, args.lr, args.slices, args.seed, w0=w0, log_every=args.log_every,
                         val_slices=zs[::4])
        t_train = time.time() - t0
        held = []
        for i in range(args.test):
            tr.add_scan(scan(9000 + i))
            held.append(tr.scans.pop())
        errs = {"base": args.base, "net": tr.rel_rmse(w, held, zs)}
        if w0 is not None:
            errs["net_at_init"] = tr.rel_rmse(w0, held, zs)
        if base is not None:
            errs["learned_linear"] = tr.rel_rmse(None, held, zs)
        tr.plan.set_taps(np.maximum(D - np.arange(D), 0) / float(D * D))
        errs["triangle"] = tr.rel_rmse(None, held, zs)
        tr.plan.set_taps(fdkod_sinc_taps(D, 2))
        errs["sinc"] = tr.rel_rmse(None, held, zs)
        if args.linear and base is None:
            # the linear learned FIR (learn.py) fitted on the same training scans
            from . import learn
            h = learn.learn(R, N, P, s, D, 2, projs, zs)
            tr.plan.set_taps(h)
            errs["learned_linear"] = tr.rel_rmse(None, held, zs)
    finally:
        tr.close()
    if args.out:
        np.save(args.out, w)
        if base is not None:
            np.save(args.out[:-4] + "_taps.npy" if args.out.endswith(".npy") else args.out + "_taps.npy", base)
    print(json.dumps({"N": N, "P": P, "s": s, "D": D, "steps": args.steps, "train_scans": args.train,
                      "held_out_scans": args.test, "train_seconds": round(t_train, 2),
                      "curve": [[int(c[0])] + [float(f"{x:.5e}") for x in c[1:]] for c in curve],
                      "rel_rmse_vs_fdk": errs}))


if __name__ == "__main__":
    main()
