"""The h-predictor network on the GPU against the FP64 oracle network at the
same BF16-rounded weights: inference, loss gradient (FP32 accumulation) and
the Adam update; features against their definition."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import need_gpu
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu


def _ctx(n=4096):
    B = need_gpu()
    return B, B.Context({}, n)


def _theta(seed=0):
    rng = np.random.default_rng(seed)
    th = rng.normal(scale=0.25, size=oracle.HNET_NPARAM).astype(np.float32)
    return th


def test_inference_matches_oracle():
    B, ctx = _ctx()
    th = _theta()
    B.sph_hnet_set_weights(ctx, th)
    X = np.random.default_rng(1).normal(size=(3001, 5)).astype(np.float32)
    X[5, 3] = 0.0
    y = B.sph_hnet_infer(ctx, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = oracle.hnet_predict(oracle.bf16_round(th), X.astype(np.float64))
    assert y[5] == 0.0
    assert np.max(np.abs(y - ref)) < 2e-5 * max(1.0, np.abs(ref).max())
    assert np.array_equal(B.sph_hnet_get_weights(ctx), th)


@pytest.mark.parametrize("nb", [1, 63, 64, 1000, 20001])
def test_gradient_matches_oracle(nb):
    B, ctx = _ctx(max(nb, 64))
    th = _theta(2)
    B.sph_hnet_set_weights(ctx, th)
    rng = np.random.default_rng(nb)
    X = rng.normal(size=(nb, 5)).astype(np.float32)
    t = rng.normal(scale=0.1, size=nb).astype(np.float32)
    loss, g = B.sph_hnet_grad(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    rl, rg = oracle.hnet_loss_grad(oracle.bf16_round(th), X.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(rl, rel=1e-4)
    assert np.max(np.abs(g - rg)) < 1e-4 * np.abs(rg).max()


def test_adam_step_matches_oracle():
    B, ctx = _ctx()
    th = _theta(3)
    B.sph_hnet_set_weights(ctx, th)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(512, 5)).astype(np.float32)
    t = rng.normal(scale=0.1, size=512).astype(np.float32)
    Xt, tt = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    _, g = B.sph_hnet_grad(ctx, Xt, tt)
    B.sph_hnet_train_step(ctx, Xt, tt, 1e-3)
    new = B.sph_hnet_get_weights(ctx)
    ref, _, _ = oracle.adam_update(th.astype(np.float64), g.astype(np.float64), np.zeros(th.size),
                                   np.zeros(th.size), 1, 1e-3)
    assert np.max(np.abs(new - ref)) < 1e-6


def test_training_reduces_loss():
    B, ctx = _ctx(8192)
    rng = np.random.default_rng(8)
    th = (rng.normal(size=oracle.HNET_NPARAM) * 0.1).astype(np.float32)
    B.sph_hnet_set_weights(ctx, th)
    X = rng.normal(size=(8192, 5)).astype(np.float32)
    t = (X[:, 3] * (0.33 - 0.1 * X[:, 4] + 0.05 * np.tanh(X[:, 0]))).astype(np.float32)
    Xt, tt = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    first = B.sph_hnet_train_step(ctx, Xt, tt, 3e-3)
    for _ in range(300):
        last = B.sph_hnet_train_step(ctx, Xt, tt, 3e-3)
    assert last < 0.05 * first


def test_features_match_definition():
    B = need_gpu()
    w = inputs.sedov(10)
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    p.hprev.copy_(p.h * 0.99)
    dt = 1e-3
    f = B.sph_hnet_features(ctx, p, dt).cpu().numpy()
    g = p.numpy()
    ref = oracle.hnet_features(g["h"], g["hprev"], g["nnb"], g["rho"], g["m"], g["divv"], dt, w.params["eta"], 1.0)
    assert np.max(np.abs(f - ref)) < 1e-5


@pytest.mark.parametrize("fp64", [True, False])
def test_step_seed_matches_oracle(fp64):
    """The fused seed of the step path (features, network and exponential in
    one tensor-core kernel) against the oracle's features and network at the
    same BF16 weights: h exp(f3 y(f)) where |f3 y| <= ln 2, else h (about 3 %
    of the particles here take that fallback)."""
    B = need_gpu()
    w = inputs.sedov(12)
    if not fp64:
        w.params["precision"] = "mixed"
    rng = np.random.default_rng(6)
    w.vx, w.vy, w.vz = 0.5 * rng.standard_normal((3, w.n))
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=fp64)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    p.hprev.copy_(p.h * torch.from_numpy(1 + 0.02 * rng.standard_normal(w.n)).to(p.h))
    th = _theta(3)
    B.sph_hnet_set_weights(ctx, th)
    dt = 0.2
    seed, fallbacks = B.sph_hnet_seed(ctx, p, dt)
    g = p.numpy()
    f = oracle.hnet_features(g["h"], g["hprev"], g["nnb"], g["rho"], g["m"], g["divv"], dt, w.params["eta"], 1.0)
    s = oracle.hnet_predict(oracle.bf16_round(th), f)
    got = seed.cpu().numpy().astype(np.float64)
    clear = np.abs(np.abs(s) - np.log(2.0)) > 1e-4          # both sides take the same branch
    inside = clear & (np.abs(s) <= np.log(2.0))
    outside = clear & (np.abs(s) > np.log(2.0))
    assert inside.sum() > 0.9 * w.n and outside.sum() > 0.01 * w.n
    assert np.max(np.abs(got[inside] / (g["h"][inside] * np.exp(s[inside])) - 1)) < 1e-4
    assert np.array_equal(got[outside], g["h"][outside])
    assert outside.sum() <= fallbacks <= w.n - inside.sum()
    # dt = 0: f3 = div v dt = 0, every particle keeps its h exactly
    seed0, fb0 = B.sph_hnet_seed(ctx, p, 0.0)
    assert fb0 == 0 and torch.equal(seed0, p.h)


def test_bounded_mma_wait_runs_out_and_the_context_is_reused():
    """With the test hook set, the tensor-core kernel issues no MMA: its 1 s
    bounded wait runs out, the call returns SPH_ERR_CUDA (no GPU fault), and
    the same context then infers correctly."""
    import time
    B, ctx = _ctx()
    th = _theta(4)
    B.sph_hnet_set_weights(ctx, th)
    X = np.random.default_rng(9).normal(size=(1000, 5)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    B.sph_test_hooks(ctx, B.SPH_TEST_SKIP_MMA)
    t0 = time.perf_counter()
    with pytest.raises(B.SphError) as e:
        B.sph_hnet_infer(ctx, Xd)
    assert e.value.code == B.SPH_ERR_CUDA and "did not complete" in str(e.value)
    assert time.perf_counter() - t0 < 30.0
    B.sph_test_hooks(ctx, 0)
    y = B.sph_hnet_infer(ctx, Xd).cpu().numpy()
    ref = oracle.hnet_predict(oracle.bf16_round(th), X.astype(np.float64))
    assert np.max(np.abs(y - ref)) < 2e-5 * max(1.0, np.abs(ref).max())
    with pytest.raises(B.SphError):
        B.sph_test_hooks(ctx, 2)
