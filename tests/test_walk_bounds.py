"""Host-side check of the free-centre forward's paired walk (index arithmetic only, no GPU).

The kernel forms a window's first and last samples as ceil(tt - k sigma / Delta) and
floor(tt + k sigma / Delta) from FP32 sums, walks NP = (floor(2 k sigma / Delta) + 4) / 2 sample pairs
from the even sample at or below the first, masks only the first pair and the last three, and
relies on two facts: the walk covers every sample of the window, and the unmasked pairs hold only
window samples.  Both are checked here in FP32 (numpy) over random phases and widths, including
widths at which 2 k sigma / Delta is within rounding of an integer."""
import numpy as np


def _window(tt, ksi):
    lo = np.ceil((tt - ksi).astype(np.float32)).astype(np.int64)     # FP32 difference, then ceil
    hi = np.floor((tt + ksi).astype(np.float32)).astype(np.int64)    # FP32 sum, then floor
    return lo, np.maximum(0, hi - lo + 1)


def test_paired_walk_covers_the_window_and_masks_enough():
    rng = np.random.default_rng(7)
    n = 2_000_000
    delta = np.float32(1500.0 / 40e6)
    inv_delta = np.float32(1.0) / delta
    k = np.float32(3.0)
    sigma = np.exp(rng.uniform(np.log(0.02e-3), np.log(0.3e-3), n)).astype(np.float32)
    # widths whose window length 2 k sigma / Delta sits within a few ulp of an integer
    m = n // 4
    target = rng.integers(4, 40, m).astype(np.float32)
    sigma[:m] = (target * delta / (2 * k)).astype(np.float32) * (1 + rng.integers(-4, 5, m) * 1.2e-7).astype(np.float32)
    ksi = (k * sigma * inv_delta).astype(np.float32)
    tt = rng.uniform(-60.0, 60.0, n).astype(np.float32)
    lo, cnt = _window(tt, ksi)
    qb = np.floor(np.float32(2) * ksi).astype(np.int64)
    NP = (qb + 4) >> 1
    assert np.all(cnt >= qb - 1) and np.all(cnt <= qb + 2)
    for off in (0, 1):                                     # parity of the window's first band row
        # every window sample (positions 0 .. cnt - 1 from the first) lies in the walk's 2 NP rows
        assert np.all(off + cnt <= 2 * NP)
        # the unmasked pairs p = 1 .. NP - 4 hold window positions 2p - off .. 2p + 1 - off only
        has_mid = NP >= 5
        last_mid = 2 * (NP - 4) + 1 - off
        assert np.all((last_mid < cnt) | ~has_mid)
        assert np.all(2 - off >= 0)
