"""The z chunk length of the single-grid step launches (host logic, no GPU).

The library cuts every tile column into z chunks, one CTA per (member, tile
column, chunk).  With `slots` CTAs resident at once, a launch of B CTAs runs in
about ceil(B / slots) rounds, each as long as one CTA's planes (its chunk plus
up to two planes beyond it).  The chosen length minimizes that product, the
longest on ties.  The pinned cases are the lengths GB300 measured fastest.
"""
import math

import numpy as np
import pytest

from paper_1705_08019_gb300 import build, fitgb


@pytest.fixture(scope="module")
def lib():
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    return fitgb.load()


def _cost(dims, tile, nmem, slots, kz):
    nx, ny, nz = dims
    cols = math.ceil(nx / tile[0]) * math.ceil(ny / tile[1])
    blocks = cols * nmem * math.ceil(nz / kz)
    return math.ceil(blocks / slots) * (kz + 2)


def test_measured_optima(lib):
    # 128^3, one member, 64x4 tiles: the FP32 step kernel (4 CTAs on each of 152 SMs)
    # was fastest with 15-plane chunks (29.6 us against 31.7 us for 8 planes), the
    # residual-field kernel (3 CTAs per SM) with 19 planes (41.2 us against 50.5 us)
    assert fitgb.fit_debug_chunk_length((128, 128, 128), (64, 4), 64, 1, 608) == 15
    assert fitgb.fit_debug_chunk_length((128, 128, 128), (64, 4), 64, 1, 456) == 19
    # 256^3 ParaExp with 16 members per launch keeps the 64-plane default
    assert fitgb.fit_debug_chunk_length((256, 256, 256), (64, 4), 64, 16, 456) == 64
    assert fitgb.fit_debug_chunk_length((256, 256, 256), (64, 4), 64, 16, 608) == 64


def test_choice_minimizes_rounds_times_planes(lib):
    rng = np.random.default_rng(3)
    for _ in range(200):
        dims = tuple(int(v) for v in rng.integers(1, 300, 3))
        tile = [(64, 4), (32, 8), (32, 4)][int(rng.integers(0, 3))]
        kz_max = int(rng.integers(1, 80))
        nmem = int(rng.integers(1, 20))
        slots = int(rng.integers(1, 1000))
        got = fitgb.fit_debug_chunk_length(dims, tile, kz_max, nmem, slots)
        top = max(1, min(kz_max, dims[2]))
        assert 1 <= got <= top
        costs = {k: _cost(dims, tile, nmem, slots, k) for k in range(1, top + 1)}
        best = min(costs.values())
        assert costs[got] == best
        assert all(costs[k] > best for k in range(got + 1, top + 1))   # the longest of the minimizers


def test_fallback_without_occupancy(lib):
    # unknown occupancy: halve from 64 while the launch has fewer than 4 x 152 CTAs
    assert fitgb.fit_debug_chunk_length((128, 128, 128), (64, 4), 64, 1, 0) == 8
    assert fitgb.fit_debug_chunk_length((256, 256, 256), (64, 4), 64, 1, 0) == 64
    assert fitgb.fit_debug_chunk_length((32, 32, 32), (32, 8), 32, 1, -1) == 8


def test_rejects_empty_sizes(lib):
    with pytest.raises(fitgb.FitError) as ei:
        fitgb.fit_debug_chunk_length((0, 4, 4), (64, 4), 64, 1, 608)
    assert ei.value.status == fitgb.FIT_ERR_ARG
