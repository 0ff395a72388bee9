"""Full-size GPU checks of the three larger synthetic workloads.

* 48^3 grid, w = 3, 4096 states, m = 24 and 64^3 grid, w = 4, 6000 states, m = 30:
  the GPU filters every column at full N (FP64 and two-float), the oracle filters
  a seeded column subset (the filter is column-independent) and the two are
  compared on those columns at 1e-12, for the FP64, two-float and Ozaki (H's 64 x 64
  blocks on the tensor cores) schedules; the GPU Lanczos bounds agree with the
  oracle's at 1e-10.
* 48^3/4096/m = 24: the two-float schedule's Ritz values (two-float filter and
  closure products), and those of the tensor-core step (Ozaki BSR filter, every step
  FP64-accurate or the first 20 with 40-bit operands, and the Ozaki closure), within
  1e-8 of the all-FP64 run's, the mixed-precision target.
* 32^3 grid, w = 2, 512 states, m = 16: the hand-written adjoint's dL/dH against
  central finite differences (h = 1e-6) of L = tr(Y^T W Y) through the GPU forward
  filter on 200 seeded random stored entries, at 1e-6 of max |dL/dH|.
"""
import numpy as np
import pytest
import torch

import chfsi_workloads as W
from tests.util import rel_fro

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


def _setup(P, oracle_mod, name):
    wl = W.workload(name)
    H = W.csr_grid(wl.g, wl.w, wl.s, wl.seed, core_frac=wl.core_frac, core_shift=wl.core_shift)
    X = W.start_block(H["N"], wl.n, wl.seed)
    v0 = W.lanczos_start(H["N"], wl.seed)
    bounds = oracle_mod.lanczos_bounds(H, v0, 20, wl.n)
    dev = torch.device("cuda")
    Hd = P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=dev)
    Xd = torch.as_tensor(X).to(dev)
    return wl, H, X, v0, bounds, Hd, Xd


@pytest.mark.parametrize("name,cols", [("g48_w3_n4096_m24", 32), ("g64_w4_n6000_m30", 24)])
def test_full_size_filter_sampled_columns(P, oracle_mod, name, cols):
    wl, H, X, v0, (a, b, a0), Hd, Xd = _setup(P, oracle_mod, name)
    dev = Xd.device
    sel = W.column_subset(wl.n, cols, wl.seed)
    Yref = oracle_mod.filter(H, X[:, sel], wl.m, a, b, a0)
    del X
    ga, gb, ga0 = P.lanczos_bounds(Hd, torch.as_tensor(v0).to(dev), 20, wl.n)
    assert abs(ga - a) <= 1e-10 * abs(a) and abs(gb - b) <= 1e-10 * abs(b) and abs(ga0 - a0) <= 1e-10 * abs(a0)
    ws = P.Workspace(dev)
    Y = torch.empty_like(Xd)
    idx = torch.as_tensor(sel, device=dev)
    for sched in (None, ["f32x2"] * wl.m):
        P.filter(Hd, Xd, wl.m, a, b, a0, schedule=sched, out=Y, workspace=ws)
        assert P.read_status(ws) == 0
        err = rel_fro(Y[:, idx].cpu().numpy(), Yref)
        assert err <= 1e-12, (sched is not None, err)
    # FP64-accurate steps with H's 64 x 64 blocks as Ozaki products, in the blocked row order
    B = W.bsr_from_csr(H, wl.g)
    perm = torch.as_tensor(B["perm"], device=dev)
    Bd = P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device=dev)
    del B
    Xp = Xd[perm].contiguous()
    Yb = torch.empty_like(Xp)
    wso = P.Workspace(dev)
    P.filter(Bd, Xp, wl.m, a, b, a0, schedule=["ozaki"] * wl.m, out=Yb, workspace=wso)
    assert P.read_status(wso) == 0
    del Xp, wso
    Y[perm] = Yb
    err = rel_fro(Y[:, idx].cpu().numpy(), Yref)
    assert err <= 1e-12, ("ozaki", err)


def test_two_float_ritz_values_meet_mixed_target_48cube(P, oracle_mod):
    """All-FP64 filter + FP64 closure against the two-float filter + two-float
    closure products: Ritz values within 1e-8 relative (max over all 4096)."""
    wl, H, X, v0, (a, b, a0), Hd, Xd = _setup(P, oracle_mod, "g48_w3_n4096_m24")
    del X
    Y = torch.empty_like(Xd)
    P.filter(Hd, Xd, wl.m, a, b, a0, out=Y)
    theta64, _ = P.rayleigh_ritz(Hd, Y, 2)
    P.filter(Hd, Xd, wl.m, a, b, a0, schedule=["f32x2"] * wl.m, out=Y)
    theta2, _ = P.rayleigh_ritz(Hd, Y, 2, precision="f32x2")
    t64, t2 = theta64.cpu().numpy(), theta2.cpu().numpy()
    assert np.all(np.diff(t64) >= 0) and np.all(np.diff(t2) >= 0)
    err = float(np.max(np.abs(t2 - t64)) / np.max(np.abs(t64)))
    assert err <= 1e-8, err


def test_ozaki_step_ritz_values_meet_mixed_target_48cube(P, oracle_mod):
    """The whole step on the tensor cores (Ozaki BSR filter steps and the Ozaki closure,
    in the blocked row order) against the all-FP64 run: Ritz values within 1e-8 relative,
    and within 1e-10 of the FP64 Ritz values' scale below the filter edge a; for every
    step FP64-accurate, and for the first 20 steps with five digit slices (40-bit
    operands) and the last 4 FP64-accurate."""
    wl, H, X, v0, (a, b, a0), Hd, Xd = _setup(P, oracle_mod, "g48_w3_n4096_m24")
    del X
    dev = Xd.device
    Y = torch.empty_like(Xd)
    P.filter(Hd, Xd, wl.m, a, b, a0, out=Y)
    theta64, _ = P.rayleigh_ritz(Hd, Y, 2)
    B = W.bsr_from_csr(H, wl.g)
    perm = torch.as_tensor(B["perm"], device=dev)
    Hp = W.permute_csr(H, B["perm"])
    Hy = P.HybridMatrix(P.CsrMatrix.from_arrays(Hp["row_ptr"], Hp["col"], Hp["val"], device=dev),
                        P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device=dev))
    del B, Hp, Hd
    Xp = Xd[perm].contiguous()
    del Xd
    t64 = theta64.cpu().numpy()
    scale = np.max(np.abs(t64))
    below = t64 < a
    for sched in (["ozaki"] * wl.m, ["ozaki40"] * (wl.m - 4) + ["ozaki"] * 4):
        P.filter(Hy, Xp, wl.m, a, b, a0, schedule=sched, out=Y)
        theta_oz, _ = P.rayleigh_ritz(Hy, Y, 2, precision="ozaki")
        toz = theta_oz.cpu().numpy()
        assert np.all(np.diff(toz) >= 0)
        err_all = float(np.max(np.abs(toz - t64)) / scale)
        err_below = float(np.max(np.abs(toz[below] - t64[below])) / scale)
        assert err_all <= 1e-8 and err_below <= 1e-10, (sched[0], err_all, err_below)


def test_adjoint_central_differences_32cube_200_entries(P, oracle_mod):
    """dL/dH from the hand-written backward against central differences of the GPU
    forward filter, 200 seeded stored entries, h = 1e-6, at 1e-6 of max |dL/dH|."""
    wl, H, X, v0, (a, b, a0), Hd, Xd = _setup(P, oracle_mod, "g32_w2_n512_m16")
    dev = Xd.device
    w = torch.as_tensor(W.loss_weights(H["N"], wl.seed)).to(dev)
    ws = P.Workspace(dev)
    Y = torch.empty_like(Xd)

    def loss():
        P.filter(Hd, Xd, wl.m, a, b, a0, out=Y, workspace=ws)
        return float(torch.sum(w[:, None] * Y * Y))

    loss()
    G = 2.0 * w[:, None] * Y
    dX, dH = P.filter_backward(Hd, Xd, G, wl.m, a, b, a0)
    dH = dH.cpu().numpy()
    scale = float(np.max(np.abs(dH)))
    rng = np.random.default_rng(wl.seed)
    picks = rng.choice(H["nnz"], 200, replace=False)
    h = 1e-6
    base = Hd.val.clone()
    worst = 0.0
    for p in picks:
        v = float(base[p])
        Hd.val[p] = v + h
        lp = loss()
        Hd.val[p] = v - h
        lm = loss()
        Hd.val[p] = v
        fd = (lp - lm) / (2.0 * h)
        worst = max(worst, abs(fd - dH[p]) / scale)
    assert torch.equal(Hd.val, base)
    assert worst <= 1e-6, worst
