"""The smoothing-length MLP on the GPU: forward and gradient of the BF16
tensor-core kernels against the FP64 oracle, training that lowers the loss,
and the learned start of the exact h iteration (fewer passes, same window)."""
import numpy as np
import pytest

import oracle as orc
from paper_2602_19873_gb300 import nl
from paper_2602_19873_gb300 import workloads as wl

from nlcheck import oracle_sorted

pytestmark = pytest.mark.gpu

BF16_RTOL = 2e-2   # BF16 operands (8-bit mantissa) in every product


def _bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16        # round to nearest even
    return r.astype(np.uint32).view(np.float32)


def _weights_as_used(P):
    """The kernels multiply BF16 weights; biases stay FP32."""
    P = P.astype(np.float64).copy()
    H, F = 64, 8
    o = 0
    for n_w, n_b in ((H * F, H), (H * H, H), (H * H, H), (H, 1)):
        P[o:o + n_w] = _bf16(P[o:o + n_w])
        o += n_w + n_b
    return P


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, 8)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 7]).astype(np.float32)
    return X, y


def test_forward_and_gradient_match_oracle():
    import torch
    X, y = _data(517, 1)                   # ragged: not a multiple of 16 or 64
    M = nl.MLP(seed=3)
    P = M.get_params()
    Pu = _weights_as_used(P)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    wd = torch.ones(len(y), dtype=torch.float32, device="cuda")
    pred = torch.empty(len(y), dtype=torch.float32, device="cuda")
    M.predict(Xd, pred)
    want = orc.mlp_forward(_bf16(X).astype(np.float64), Pu)
    got = pred.cpu().numpy()
    assert np.max(np.abs(got - want)) <= BF16_RTOL * (np.abs(want).max() + 1.0)
    g = torch.empty(M.nparams(), dtype=torch.float32, device="cuda")
    loss = M.grad(Xd, yd, wd, g)
    lw, gw = orc.mlp_loss_grad(_bf16(X).astype(np.float64), y.astype(np.float64), Pu)
    assert abs(loss - lw) <= BF16_RTOL * lw
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - gw) <= BF16_RTOL * np.linalg.norm(gw)
    # every layer's block separately (a transposed operand would fail here)
    H, F = 64, 8
    o = 0
    for n_blk in (H * F, H, H * H, H, H * H, H, H, 1):
        a, b = gg[o:o + n_blk], gw[o:o + n_blk]
        assert np.linalg.norm(a - b) <= 3 * BF16_RTOL * (np.linalg.norm(b) + 1e-12), o
        o += n_blk
    M.free()


def test_training_lowers_the_loss():
    import torch
    X, y = _data(20000, 2)
    M = nl.MLP(seed=5)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    wd = torch.ones(len(y), dtype=torch.float32, device="cuda")
    g = torch.empty(M.nparams(), dtype=torch.float32, device="cuda")
    l0 = M.grad(Xd, yd, wd, g)
    l1 = M.train(Xd, yd, wd, epochs=15, batch=2048, lr=3e-3, seed=1)
    assert l1 < 0.2 * l0, (l0, l1)
    # checkpoint round trip
    P = M.get_params()
    M2 = nl.MLP(seed=9)
    M2.set_params(P)
    a = torch.empty(len(y), dtype=torch.float32, device="cuda")
    b = torch.empty(len(y), dtype=torch.float32, device="cuda")
    M.predict(Xd, a)
    M2.predict(Xd, b)
    assert torch.equal(a, b)
    M.free()
    M2.free()


def _converged(d, start, mlp=None):
    import torch
    t = {k: torch.from_numpy(d[k]).cuda() for k in ("x", "y", "z", "h")}
    p = nl.make_params(key=1, cluster=8, support=2.0)
    L = nl.NeighborList()
    if mlp is not None:
        L.set_mlp(mlp)
    h = t["h"].clone()
    info = L.iterate_h(t["x"], t["y"], t["z"], h, d["box"], p, 100.0, 2.0, max_iter=80,
                       start=start)
    return L, h, info


def test_learned_start_needs_fewer_passes():
    import torch
    mlp = nl.MLP(seed=11)
    Xs, ys, ws = [], [], []
    for seed in range(4):                       # training systems
        d = wl.plummer(60000, n_spheres=6, seed=600 + seed, n_target=100)
        L, h, info = _converged(d, nl.NL_HSTART_PLAIN)
        X, e64 = L.mlp_features()
        y, w = L.mlp_targets(h, e64)
        Xs.append(X), ys.append(y), ws.append(w)
        L.free()
    X, y, w = torch.cat(Xs), torch.cat(ys), torch.cat(ws)
    loss = mlp.train(X, y, w, epochs=40, batch=2048, lr=3e-3, seed=2)
    assert loss < 0.1
    d = wl.plummer(120000, n_spheres=8, seed=700, n_target=100)     # evaluation system
    Lp, hp, ip = _converged(d, nl.NL_HSTART_PLAIN)
    Ll, hl, il = _converged(d, nl.NL_HSTART_LEARNED, mlp)
    assert ip["unconverged"] == 0 and il["unconverged"] == 0
    assert il["iterations"] < ip["iterations"], (il, ip)
    # the learned start does not change what is accepted: the window holds
    hc = hl.cpu().numpy()
    q = np.random.default_rng(0).integers(0, len(hc), 64)
    cnt = orc.gather_counts_brute(d["x"], d["y"], d["z"], hc, d["box"], 2.0, q)
    assert np.abs(cnt - 100).max() <= 2
    Lp.free()
    Ll.free()
    mlp.free()


# Features and targets are logs of ratios of FP32 box sides and of mean h:
# each ratio carries a few FP32 roundings (relative 2^-23 each, about 2.4e-7
# in the log) and logf adds 2 ulp of its result (|log| <= 20: about 4e-6).
FEATURE_ATOL = 1e-5


@pytest.mark.parametrize("name,M", [("plummer", 8), ("uniform", 8), ("evrard", 16),
                                    ("plummer", 4)])
def test_features_and_targets_match_oracle(name, M):
    """Per-cluster features and training targets of the learned start,
    element by element against the FP64 oracle on the oracle's own sort of
    the same particles (ragged sizes: partly filled last super-clusters)."""
    import torch
    d = {"plummer": lambda: wl.plummer(30011, n_spheres=4, seed=41),
         "uniform": lambda: wl.uniform(20005, seed=42),
         "evrard": lambda: wl.evrard(25003, seed=43)}[name]()
    o = oracle_sorted(d)
    Xw, e64w = orc.mlp_features(o["xs"], o["ys"], o["zs"], d["box"], M)
    yw, ww = orc.mlp_targets(o["hs"], M, e64w)
    t = {k: torch.from_numpy(np.ascontiguousarray(d[k], dtype=np.float32)).cuda()
         for k in ("x", "y", "z", "h")}
    p = nl.make_params(key=d["kind"], cluster=M, support=d["support"])
    L = nl.NeighborList().build(t["x"], t["y"], t["z"], t["h"], d["box"], p)
    X, e64 = L.mlp_features()
    y, w = L.mlp_targets(t["h"], e64)
    torch.cuda.synchronize()
    X, e64, y, w = (a.cpu().numpy().astype(np.float64) for a in (X, e64, y, w))
    assert X.shape == Xw.shape and e64.shape == e64w.shape
    assert np.max(np.abs(e64 - e64w) / e64w) <= 1e-6
    err = np.abs(X - Xw)
    assert err.max() <= FEATURE_ATOL, (np.unravel_index(err.argmax(), err.shape), err.max())
    assert np.array_equal(w, ww)
    assert np.max(np.abs(y - yw)) <= FEATURE_ATOL
    L.free()
