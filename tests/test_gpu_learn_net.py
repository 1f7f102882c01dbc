"""Training of the learned decimation with the library's kernels
(paper_1708_07515_gb300.learn_net) on a small scan: the relative error of
FDK-OD against full FDK on the training slices falls, and the trained net
keeps a held-out scan at least as close to full FDK as the plain low-pass."""
import numpy as np
import pytest

import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    fd.load()
    return fd


def test_training_reduces_the_error_against_full_fdk(fd):
    from paper_1708_07515_gb300 import learn_net
    N, P, s, D = 48, 96, 2, 4
    R = 4.0 * N
    tr = learn_net.Trainer(R, N, P, s, D)
    try:
        for i in range(2):
            tr.add_scan(phantom.project_gpu(phantom.make_phantom(7000 + i, N, 10), R, N, N, P))
        zs_eval = np.arange(6, N - 6, 4)
        before = tr.rel_rmse(None, tr.scans, zs_eval)
        w, curve = learn_net.train(tr, steps=60, lr=3e-3, slices=4, seed=3, log_every=1)
        after = tr.rel_rmse(w, tr.scans, zs_eval)
        tr.add_scan(phantom.project_gpu(phantom.make_phantom(7100, N, 10), R, N, N, P))
        held = [tr.scans.pop()]
        held_plain = tr.rel_rmse(None, held, zs_eval)
        held_net = tr.rel_rmse(w, held, zs_eval)
    finally:
        tr.close()
    losses = np.array([c[1] for c in curve])
    assert np.isfinite(losses).all()
    assert losses[-10:].mean() < 0.9 * losses[:3].mean(), losses
    assert after < before, (before, after)
    assert held_net <= held_plain * 1.02, (held_plain, held_net)
