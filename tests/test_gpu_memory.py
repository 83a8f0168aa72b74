"""ParaExp members per pass chosen from the free device memory.

With opts.members_per_pass = 0 the library advances all K members together
unless their states do not fit in the device memory left; then it runs them
in passes of as many members as fit.  The test takes most of the device memory
with a torch allocation so that about three members' states fit, and checks
that the solve then runs in several passes (more step launches) and gives the
same bits as the all-at-once solve (members are independent and the
superposition order is fixed).
"""
import numpy as np
import pytest

import oracle
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _launches(lengths, mpp):
    """Step launches of a solve in passes of at most mpp members: members
    ordered by decreasing length and grouped from the shortest end, the first
    (shortest) group taking the remainder; each pass runs to its longest
    member's length."""
    order = sorted(lengths, reverse=True)
    n = len(order)
    npass = -(-n // mpp)
    total, end = 0, n
    for p in range(npass):
        first = end - (n - (npass - 1) * mpp if p == 0 else mpp)
        total += order[first]
        end = first
    return total


def test_members_per_pass_follow_free_memory():
    import torch
    w = W.small_random(dims=(96, 64, 48), nsteps=160, K=8, seed=5, precision=32)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    win = w.windows()
    lengths = [int(win[-1] - win[j]) for j in range(w.K)]
    g = fitgb.Grid.from_workload(w, 32)
    ref = g.paraexp(dt, w.K, win, w.sources, w.probes)
    assert fitgb.fit_last_stats(g.handle)["step_launches"] == max(lengths)
    # explicit groups of three: the partition the launch count model describes
    got3 = g.paraexp(dt, w.K, win, w.sources, w.probes, opts=fitgb.make_opts(members_per_pass=3))
    assert fitgb.fit_last_stats(g.handle)["step_launches"] == _launches(lengths, 3)
    for a, b in zip(ref, got3):
        assert np.array_equal(a, b)
    g.close()

    nx, ny, nz = w.dims
    ncp = ((nx + 3) // 4 * 4) * ny * nz
    per = 2 * 6 * 4 * ncp            # one member: e and h, two time levels, FP32
    coef = 2 * 3 * 4 * ncp           # ca and cb, taken before the member count is chosen
    g = fitgb.Grid.from_workload(w, 32)
    free, total = torch.cuda.mem_get_info()
    margin = (1 << 30) + total // 64
    target = margin + int(3.5 * per) + coef   # about three and a half members' states left
    assert free > target + (1 << 30)
    hog = torch.empty(free - target, dtype=torch.uint8, device="cuda")
    try:
        got = g.paraexp(dt, w.K, win, w.sources, w.probes)
        launches = fitgb.fit_last_stats(g.handle)["step_launches"]
    finally:
        del hog
        torch.cuda.empty_cache()
        g.close()
    mpp = [m for m in range(1, w.K + 1) if _launches(lengths, m) == launches]
    assert mpp and 2 <= mpp[0] <= 4, (launches, mpp)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
