"""The learned warm start against the method without it: a U-Net trained on phantom/signal pairs
that the forward operator generates must let the reconstruction reach the plain reconstruction's
final residual (from zero, 50 iterations, its best step size) within a relative 1e-3, in less
device time.  Small training set (CI-sized); the full 2000/200-seed run is
`python -m paper_2602_03893_gb300.warmstart`."""
import pytest

from paper_2602_03893_gb300 import warmstart

pytestmark = pytest.mark.gpu


def test_warm_start_beats_plain_reconstruction():
    rep, _ = warmstart.run(n_train=96, n_eval=3, n_timed=2, epochs=2, lr=1e-3, iters=50, procs=4, log=None,
                           etas=(0.02, 0.05, 0.1))
    assert rep["train_loss_last"] < 0.1 * rep["train_loss_first"]
    assert rep["reached_frac"] == 1.0
    assert rep["warm_s_mean"] < rep["plain_s_mean"]
    for r in rep["rows"]:
        assert r["warm_resid"] <= (1 + 1e-3) * r["plain_resid"]
