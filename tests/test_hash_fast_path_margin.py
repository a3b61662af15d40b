"""The bucket hash's FP32 fast path (gsph_internal.cuh, bucket_coord_fast) restated in numpy: the
coordinate truncated to FP32 from its bits, the FP32 difference and product, and the margin
2^-22 (|tf| + 1 + (|x| + |lo|) / 2h). Outside the margin its floor must equal the FP64 definition
floor(fl64(fl64(x - lo) / 2h)) (Sec. I bucket hash) for every input: values a few thousand ulps from every
bucket face of the Taylor bar's and the collapse block's grids, random values inside them, and the
special inputs that must take the FP64 path."""
import numpy as np

from paper_2310_03596_gb300 import scenes


def trunc32(x):
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    e = ((hi >> np.uint32(20)) & np.uint32(0x7FF)).astype(np.int64)
    ok = (e >= 1023 - 126) & (e <= 1023 + 127)
    bits = ((hi & np.uint32(0x80000000)) | ((e - 896).clip(0, 255).astype(np.uint32) << np.uint32(23))
            | ((hi & np.uint32(0xFFFFF)) << np.uint32(3)) | (lo >> np.uint32(29)))
    return bits.view(np.float32), ok


def fast_path(x, lo, cell, dim):
    """(decided, coordinate) of the FP32 fast path, FP32 arithmetic rounded as on the GPU."""
    inv = np.float32(1.0 / cell)
    xt, ok = trunc32(x)
    lof = np.float32(lo)
    with np.errstate(all="ignore"):
        df = (xt - lof).astype(np.float32)
        tf = (df * inv).astype(np.float32)
        fl = np.floor(tf)
        fr = (tf - fl).astype(np.float32)
        span = ((np.abs(xt) + np.abs(lof)).astype(np.float32) * inv).astype(np.float32)
        eps = (np.float32(2.0 ** -22) * ((np.abs(tf) + np.float32(1)).astype(np.float32) + span)).astype(np.float32)
        decided = ok & (fr > eps) & (fr < (np.float32(1) - eps)) & (np.abs(df) >= np.float32(2.0 ** -126))
        got = np.where(fl < 0, -1, np.where(fl >= dim, dim, np.nan_to_num(fl))).astype(np.int64)
    return decided, got


def definition(x, lo, cell, dim):
    with np.errstate(all="ignore"):
        t = np.floor((x - lo) / cell)
    return np.where(~(t >= 0), -1, np.where(t >= dim, dim, np.nan_to_num(t))).astype(np.int64)


def test_fast_path_agrees_with_the_fp64_definition():
    rng = np.random.default_rng(7)
    checked = 0
    for sc in (scenes.taylor_bar(), scenes.collapse_block(dx=2e-3)):
        cell = 2.0 * sc.h
        for a in range(3):
            lo, dim = float(sc.grid_lo[a]), int(sc.grid_dims[a])
            faces = lo + np.arange(dim + 1) * cell
            near = faces[:, None] + rng.integers(-3000, 3000, (faces.size, 64)) * np.spacing(faces)[:, None]
            inside = lo + rng.random(20000) * dim * cell
            x = np.concatenate([near.ravel(), inside])
            decided, got = fast_path(x, lo, cell, dim)
            want = definition(x, lo, cell, dim)
            assert np.array_equal(got[decided], want[decided])
            # values off the faces almost all take the fast path
            assert decided[near.size:].mean() > 0.99
            checked += int(decided.sum())
    assert checked > 100000


def test_special_inputs_take_the_fp64_path():
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-300, 1e300, 5e-39])
    decided, _ = fast_path(x, 0.0, 3.25e-4, 100)
    assert not decided.any()
