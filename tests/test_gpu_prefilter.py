"""GPU tests of the learned prefilter: its forward and backward kernels against a NumPy
float32 reference computed on the same bf16-rounded operands (logits within 1e-2
absolute; gradients to float32 accumulation-order accuracy), learning on a rule it can
represent, bit-identical resume from a checkpoint, selection and the feature kernel."""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu
MAT = synth.blosum62()


@pytest.fixture(scope="module")
def env():
    import paper_2009_14467_gb300 as P
    from paper_2009_14467_gb300 import prefilter as F
    ctx = P.Context(0)
    yield P, F, ctx
    ctx.close()


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def cpu_forward(net, x):
    w1, b1 = net.w1b.float().cpu().numpy(), net.b1.cpu().numpy()
    w2, b2 = net.w2b.float().cpu().numpy(), net.b2.cpu().numpy()
    w3, b3 = net.w3b.float().cpu().numpy(), net.b3.cpu().numpy()
    h1 = bf16(np.maximum(x @ w1 + b1, 0))
    h2 = bf16(np.maximum(h1 @ w2 + b2, 0))
    z = h2 @ w3 + b3[0]
    return h1, h2, z, (w1, w2, w3)


def test_logits_match_cpu_reference(env):
    P, F, ctx = env
    net = F.MLP(seed=3)
    rng = np.random.default_rng(0)
    x = bf16(rng.normal(size=(5000, 16)))
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    z = F.forward(ctx, net, xd).cpu().numpy()
    _, _, zc, _ = cpu_forward(net, x)
    assert np.abs(z - zc).max() <= 1e-2
    assert np.abs(z - zc).max() <= 1e-3 * max(1.0, np.abs(zc).max())


def test_gradients_match_cpu_reference(env):
    P, F, ctx = env
    net = F.MLP(seed=4)
    rng = np.random.default_rng(1)
    n = 96
    x = bf16(rng.normal(size=(n, 16)))
    y = (rng.random(n) < 0.3).astype(np.float32)
    pw = 3.0
    F.train_step(ctx, net, torch.from_numpy(x).to(torch.bfloat16).cuda(), torch.from_numpy(y).cuda(), 0.0, pw)
    g = [t.cpu().numpy() for t in net.grads()]
    h1, h2, z, (w1, w2, w3) = cpu_forward(net, x)
    wt = np.where(y > 0.5, pw, 1.0)
    dz = wt * (1 / (1 + np.exp(-z)) - y) / n
    gw3 = h2.T @ dz
    gb3 = dz.sum()
    dpre2 = bf16(np.where(h2 > 0, dz[:, None] * w3[None, :], 0))
    gw2 = h1.T @ dpre2
    gb2 = dpre2.sum(0)
    dh1 = dpre2 @ w2.T
    gb1 = np.where(h1 > 0, dh1, 0).sum(0)
    dpre1 = bf16(np.where(h1 > 0, dh1, 0))
    gw1 = x.T @ dpre1
    for got, want in zip(g, [gw1, gb1, gw2, gb2, gw3, np.array([gb3])]):
        scale = max(np.abs(want).max(), 1e-12)
        assert np.abs(got - want).max() <= 2e-3 * scale


def test_training_learns_and_resume_is_bit_identical(env):
    P, F, ctx = env
    rng = np.random.default_rng(2)
    n = 40000
    x = bf16(rng.normal(size=(n, 16)))
    y = ((x[:, 0] + 0.5 * x[:, 9] - 0.3 * x[:, 4]) > 0.8).astype(np.float32)
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    yd = torch.from_numpy(y).cuda()
    net = F.MLP(seed=5)
    h = F.train(ctx, net, xd, yd, epochs=2, batch=4096, lr=3e-3, seed=9)
    assert h[-1] < h[0]
    z = F.forward(ctx, net, xd).cpu().numpy()
    acc = ((z > 0) == (y > 0.5)).mean()
    assert acc > 0.95
    # resume: a copy taken now and trained one more epoch matches the original
    sd = net.state_dict()
    twin = F.MLP(seed=123)
    twin.load_state_dict(sd)
    F.train(ctx, net, xd, yd, epochs=1, batch=4096, lr=3e-3, seed=10)
    F.train(ctx, twin, xd, yd, epochs=1, batch=4096, lr=3e-3, seed=10)
    for k in ("w1", "w2", "w3", "b1", "b2", "b3", "adam_m", "adam_v"):
        assert torch.equal(getattr(net, k), getattr(twin, k)), k


def test_select_keeps_logits_above_threshold(env):
    P, F, ctx = env
    n = 10007
    rng = np.random.default_rng(3)
    pairs = np.zeros(n, P.CAND_DTYPE)
    pairs["i"] = np.arange(n)
    pairs["j"] = np.arange(n) + 1
    z = rng.normal(size=n).astype(np.float32)
    out = F.select(ctx, torch.from_numpy(pairs.view(np.uint8).reshape(n, 20)).cuda(), torch.from_numpy(z).cuda(), 0.25)
    got = P.to_records(out, P.CAND_DTYPE)
    assert (got["i"] == np.flatnonzero(z >= 0.25)).all()


def test_features_match_formula(env):
    P, F, ctx = env
    ps = synth.families_1k().subset(np.arange(200))
    codes = O.encode(ps.ascii)
    rp, code, pos = O.kmers(codes, ps.offsets, 6)
    c = O.candidates(rp, code, pos, 6, 0, MAT, 1)
    x = F.features(ctx, torch.from_numpy(codes).cuda(), torch.from_numpy(ps.offsets).cuda(),
                   torch.from_numpy(c.view(np.uint8).reshape(-1, 20)).cuda(), P.Params(matrix=MAT))
    x = x.float().cpu().numpy()
    L = np.diff(ps.offsets)
    for r, rec in enumerate(c[:50]):
        li, lj = float(L[rec["i"]]), float(L[rec["j"]])
        qi, tj = ps.offsets[rec["i"]], ps.offsets[rec["j"]]
        two = rec["qpos"][1] != 0xFFFF
        s0 = sum(int(MAT[codes[qi + rec["qpos"][0] + t], codes[tj + rec["tpos"][0] + t]]) for t in range(6))
        s1 = sum(int(MAT[codes[qi + rec["qpos"][1] + t], codes[tj + rec["tpos"][1] + t]]) for t in range(6)) if two else 0
        d0 = float(rec["qpos"][0]) - float(rec["tpos"][0])
        d1 = float(rec["qpos"][1]) - float(rec["tpos"][1]) if two else d0
        mn, mx = min(li, lj), max(li, lj)
        want = [np.log1p(rec["count"]), d0 / 256, d1 / 256, abs(d0 - d1) / 256, np.log(li + 1), np.log(lj + 1),
                np.log(mn + 1), np.log(mx + 1), mn / mx, s0 / 32, s1 / 32, (s0 + s1) / 32, rec["count"] / mn,
                1.0 if two else 0.0, 0, 0]
        np.testing.assert_allclose(x[r], bf16(want), rtol=1e-2, atol=1e-3)
