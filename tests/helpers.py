"""Shared helpers of the device parity tests (inputs from ``synth``, expectations from ``oracle``)."""
import os

import numpy as np
import pytest

FWD_ATOL = 1e-4   # forward image: max abs error per channel (fp32 kernels vs binary64 oracle)
GRAD_RTOL = 1e-3  # gradients: |g - g*| <= 1e-3 max(|g*|, 1e-3 max_col |g*|) + SUM_RTOL A*
# A* = sum over pixels of |one pixel's contribution| (from the oracle).  A gradient is a sum of
# per-pixel terms, each computed in binary32 with a small relative error; when the terms cancel,
# that error is relative to A*, not to the sum.  2D terms carry ~1e-6 relative error; in 3D the
# transmittance in front of a layer of opacity a is recovered by dividing by 1 - a, so an alpha
# error of ~1e-6 becomes ~1e-6 / (1 - a) <= 1e-4 relative.
# In 2D no entry needs it (every 2D gradient entry passes the plain check), so it is 0 there.
SUM_RTOL = {2: 0.0, 3: 2e-4}
# Gradient entries must pass the plain check |g - g*| <= 1e-3 max(|g*|, floor), without the
# summation-scale term, in at least this share of every column; the rest are counted and reported.
PLAIN_PASS = 0.999
# Largest share of pixels whose threshold decisions (alpha_min skip, T_min stop) lie within the
# kernels' error bound of their threshold (the oracle's ambiguity bits); such pixels are excluded
# from the forward check and carry no upstream gradient in the backward check.
AMB_SHARE = 1e-3

# (kind, test, detail, value, limit) rows printed in the terminal summary (tests/conftest.py)
REPORT = []


def _label():
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0].split("::", 1)[-1]


def check_amb_share(amb, what="image", limit=AMB_SHARE):
    """Assert and report the share of ambiguous pixels."""
    share = float(np.mean(amb)) if np.size(amb) else 0.0
    REPORT.append(("ambiguous share", _label(), what, share, limit))
    assert share < limit, (what, share, limit)
    return share


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib_ready():
    from paper_2508_12615_gb300 import build

    build.build()
    import paper_2508_12615_gb300 as w

    return w


# Per-column counts of the plain check pooled over several cases: pool name -> column -> [entries,
# entries that need the summation term]
POOL = {}


def grad_close(g, ref, gabs=None, dims=2, rtol=GRAD_RTOL, floor_frac=1e-3, cols=None, pool=None):
    """Column-floored relative check with the summation-scale term; returns (ok, worst ratio, index).
    The plain pass rate (without the summation term) must reach PLAIN_PASS in every column of this
    case; with `pool` given, the column counts are pooled under that name instead and checked by
    check_pooled_plain_rate (for columns of a few hundred entries, a share of 1e-3 is below one
    entry)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    gabs = np.zeros_like(ref) if gabs is None else np.asarray(gabs, np.float64)
    if cols is not None:
        g, ref, gabs = g[:, cols], ref[:, cols], gabs[:, cols]
    floor = floor_frac * np.abs(ref).max(axis=0, keepdims=True)
    plain = rtol * np.maximum(np.abs(ref), floor)
    err = np.abs(g - ref)
    tol = plain + SUM_RTOL[dims] * gabs
    ratio = err / np.maximum(tol, 1e-30)
    idx = np.unravel_index(np.argmax(ratio), ratio.shape)
    # entries that pass without the summation-scale term, per column
    rate = (err <= plain).mean(axis=0) if g.shape[0] else np.ones(g.shape[1])
    worst_col = int(np.argmin(rate))
    n_sum_only = int((err > plain).sum())
    col = cols[worst_col] if cols is not None else worst_col
    REPORT.append(("plain 1e-3 pass rate", _label(), f"min over columns (col {col}; {n_sum_only} of {err.size} "
                   f"entries need the summation term)", float(rate.min()), PLAIN_PASS))
    if pool is not None:
        p = POOL.setdefault(pool, {})
        for k in range(err.shape[1]):
            c = cols[k] if cols is not None else k
            n_k, f_k = p.get(c, (0, 0))
            p[c] = (n_k + err.shape[0], f_k + int((err[:, k] > plain[:, k]).sum()))
        ok = bool(np.all(ratio <= 1.0))
    else:
        ok = bool(np.all(ratio <= 1.0)) and bool(rate.min() >= PLAIN_PASS)
    return ok, float(ratio.max()), (idx, "plain pass rate", float(rate.min()), "column", col)


def check_pooled_plain_rate(pool):
    """Assert and report, per column, the plain pass rate pooled over the cases recorded under `pool`."""
    p = POOL.get(pool)
    if not p:
        pytest.skip(f"no case recorded under {pool!r} in this session")
    rates = {c: 1.0 - f / n for c, (n, f) in p.items() if n}
    worst = min(rates, key=rates.get)
    n_tot = sum(n for n, _ in p.values())
    f_tot = sum(f for _, f in p.values())
    REPORT.append(("plain 1e-3 pass rate", _label(), f"pooled '{pool}', min over columns (col {worst}; "
                   f"{f_tot} of {n_tot} entries need the summation term)", rates[worst], PLAIN_PASS))
    assert rates[worst] >= PLAIN_PASS, (pool, worst, p[worst])


def sample_pixels(H, W, n, seed):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, W, n)
    v = rng.integers(0, H, n)
    # always include the image corners and the last ragged tile
    extra = np.array([[0, 0], [W - 1, 0], [0, H - 1], [W - 1, H - 1]])
    return np.concatenate([np.stack([u, v], 1), extra]).astype(np.int32)
