"""The bound behind the FP32 screen of the OC bisection candidates.

For each candidate the OC kernel first sums the clamped volumes
t = max(min(ocP / lmid, hi), lo) in FP32 (ocP, 1/lmid and the move limits
rounded to FP32, per-thread sequential FP32 sums of at most M terms, then FP64
across threads). It trusts a bisection decision only when the screened sum is
farther from the threshold than

    nact (4.01 u + 2e-15) + 1.01 (M - 1) u |S32|,   u = 2^-24,

and redoes the pass in FP64 otherwise. The bound must therefore cover
|S32 - sum of the FP64 terms| for every input the screen accepts
(1e-30 <= lmid <= 1e30): here the FP32 arithmetic is emulated in numpy
(IEEE float32, round to nearest, the same operation order) on designs whose
ocP runs from float32-subnormal to beyond the float32 range, and the FP64
terms are summed exactly (math.fsum)."""
import math

import numpy as np
import pytest

U = 2.0 ** -24


def _screen(x, ocp, move, inv, threads):
    n = len(x)
    with np.errstate(over="ignore"):
        o32 = ocp.astype(np.float32)  # beyond the float32 range: inf, clamped to hi like the FP64 term
    hi64, lo64 = np.minimum(x + move, 1.0), np.maximum(x - move, 0.0)
    hi32, lo32 = hi64.astype(np.float32), lo64.astype(np.float32)
    with np.errstate(over="ignore", under="ignore"):
        t32 = np.maximum(np.minimum(o32 * np.float32(inv), hi32), lo32)
    M = -(-n // threads)
    pad = np.zeros(M * threads, np.float32)
    pad[:n] = t32
    acc = np.zeros(threads, np.float32)
    for row in pad.reshape(M, threads):  # thread j sums elements j, j + threads, ... in order
        acc = (acc + row).astype(np.float32)
    s32 = math.fsum(acc.astype(np.float64))
    t64 = np.maximum(np.minimum(ocp * inv, hi64), lo64)
    return s32, math.fsum(t64), M


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("threads", [7, 64, 1000])
def test_fp32_screen_within_bound(seed, threads):
    rng = np.random.default_rng(seed)
    n = 5000
    x = np.clip(rng.random(n) * 1.2 - 0.1, 0.0, 1.0)
    lg = rng.uniform(-45, 45, n) if seed % 2 else rng.uniform(-3, 3, n)
    ocp = x * 10.0 ** lg
    ocp[rng.random(n) < 0.05] = 0.0
    move = [0.2, 0.05, 1.0][seed % 3]
    med = float(np.median(ocp[ocp > 0]))
    for inv in [1e-30, 1e30, 1.0, 1.0 / med, 3.7 / med, 0.21 / med, float(rng.uniform(0.5, 2.0)) / med]:
        if not (1e-30 <= inv <= 1e30):
            continue
        s32, s64, M = _screen(x, ocp, move, inv, threads)
        bound = n * (4.01 * U + 2e-15) + 1.01 * (M - 1) * U * abs(s32)
        assert abs(s32 - s64) <= bound, (inv, s32, s64, bound)


def test_bound_is_not_vacuous():
    """At the bench's scale the bound is far below the volume step of a late
    bisection decision, so the screen decides almost every pass in FP32."""
    n, vol = 221184, 0.12
    bound = n * (4.01 * U + 2e-15) + 1.01 * 2 * U * n * vol
    assert bound / n < 5e-7  # a decision at a 1e-4 bracket moves the mean volume by ~1e-5
