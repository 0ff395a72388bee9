"""Full-size runs of the two largest synthetic workloads (opt-in: they take
minutes; set CHFSI_SCALE_TESTS=1).  The GPU filters every column at full N; the
oracle filters a seeded column subset (the filter is column-independent) and
the two are compared on those columns."""
import os

import numpy as np
import pytest
import torch

import chfsi_workloads as W
from tests.util import rel_fro

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("CHFSI_SCALE_TESTS") != "1",
                                 reason="opt-in full-size runs (CHFSI_SCALE_TESTS=1)")]


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


@pytest.mark.parametrize("name,cols", [("g48_w3_n4096_m24", 32), ("g64_w4_n6000_m30", 24)])
def test_full_size_filter_sampled_columns(P, oracle_mod, name, cols):
    wl = W.workload(name)
    H = W.csr_grid(wl.g, wl.w, wl.s, wl.seed, core_frac=wl.core_frac, core_shift=wl.core_shift)
    X = W.start_block(H["N"], wl.n, wl.seed)
    v0 = W.lanczos_start(H["N"], wl.seed)
    a, b, a0 = oracle_mod.lanczos_bounds(H, v0, 20, wl.n)
    dev = torch.device("cuda")
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    Xd = torch.as_tensor(X).to(dev)
    sel = W.column_subset(wl.n, cols, wl.seed)
    Yref = oracle_mod.filter(H, X[:, sel], wl.m, a, b, a0)
    # Lanczos bounds on the GPU agree with the oracle's
    ga, gb, ga0 = P.lanczos_bounds(Hd, torch.as_tensor(v0).to(dev), 20, wl.n)
    assert abs(ga - a) <= 1e-10 * abs(a) and abs(gb - b) <= 1e-10 * abs(b) and abs(ga0 - a0) <= 1e-10 * abs(a0)
    ws = P.Workspace(dev)
    Y = torch.empty_like(Xd)
    for sched, tol in ((None, 1e-12), (["f32x2"] * wl.m, 1e-12)):
        P.filter(Hd, Xd, wl.m, a, b, a0, schedule=sched, out=Y, workspace=ws)
        assert P.read_status(ws) == 0
        Ys = Y[:, torch.as_tensor(sel, device=dev)].cpu().numpy()
        assert rel_fro(Ys, Yref) <= tol, sched
