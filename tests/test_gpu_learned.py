"""The learned classifier on the GPU (params.classify = BSPS_LEARNED).

* loss and gradient of the GPU kernels vs the float64 CPU oracle (oracle/mlp.py),
  relative error <= 1e-3 (FP32 accumulation over <= 16384 points);
* sorts with the learned classifier are bit-identical to the oracle (keys,
  payloads, bucket sizes, splitters, per-key buckets): the correction makes the
  bucket exact whatever the network predicts;
* the classifier's evaluation of the network (piecewise affine through the
  first layer's knots) against the oracle's plain forward pass;
* what training and the index over the network's output gain: the loss
  never rises above the spline start's, and keys need few splitter
  comparisons.
"""
import math

import numpy as np
import pytest

import bsp_inputs as gen
import oracle
from oracle import mlp
from tests.gpu_util import assert_same, lib, run_gpu

pytestmark = pytest.mark.gpu


def _theta(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.4, mlp.N_PARAMS).astype(np.float32)


@pytest.mark.parametrize("m", [1, 100, 4096, 16384])
def test_gradient_matches_oracle(m):
    import torch
    bsps = lib()
    rng = np.random.default_rng(m)
    x = np.sort(rng.random(m)).astype(np.float32)
    y = ((np.arange(m) + 0.5) / m).astype(np.float32)
    theta = _theta(m)
    dev = "cuda:0"
    tp, tx, ty = (torch.from_numpy(a).to(dev) for a in (theta, x, y))
    grad = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ws = torch.empty(bsps.bsps_mlp_workspace_size(m), dtype=torch.uint8, device=dev)
    assert bsps.bsps_mlp_loss_grad(tp, tx, ty, m, grad, loss, ws) == 0
    torch.cuda.synchronize()
    ref_loss, ref_grad = mlp.loss_and_grad(theta.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ref_loss) <= 1e-3 * abs(ref_loss) + 1e-9
    scale = np.abs(ref_grad).max()
    assert np.abs(g - ref_grad).max() <= 1e-3 * scale + 1e-9


@pytest.mark.parametrize("kind", ["random", "spline"])
def test_piecewise_affine_evaluation_matches_oracle_forward(kind):
    """The classifier evaluates the network through its first layer's knots
    (layer 2 affine between consecutive knots); it must give the oracle's
    plain forward pass: random parameters of both signs, and a spline start,
    at points inside and outside [0, 1] and exactly on knots."""
    import torch
    bsps = lib()
    rng = np.random.default_rng(17)
    if kind == "random":
        theta = _theta(3)
    else:
        px = np.sort(rng.random(5000))
        py = (np.arange(5000) + 0.5) / 5000
        theta = mlp.spline_start(px, py)[0].astype(np.float32)
    W1, b1 = theta[:32], theta[32:64]
    on = W1 != 0
    knots = (-b1[on] / W1[on]).astype(np.float32)
    x = np.concatenate([rng.random(20000) * 1.4 - 0.2, knots, np.linspace(-2, 3, 101)]).astype(np.float32)
    dev = "cuda:0"
    tp, tx = torch.from_numpy(theta).to(dev), torch.from_numpy(x).to(dev)
    ty = torch.empty_like(tx)
    ws = torch.empty(bsps.bsps_mlp_workspace_size(0), dtype=torch.uint8, device=dev)
    assert bsps.bsps_mlp_predict(tp, tx, x.shape[0], ty, ws) == 0
    ref, (_, z1, h1, z2, h2) = mlp.forward(theta.astype(np.float64), x.astype(np.float64))
    # FP32 against float64: the bound scales with the magnitude of the terms summed
    scale = 1.0 + np.abs(h2) @ np.abs(theta[-33:-1].astype(np.float64))
    err = np.abs(ty.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 1e-5 * scale), float((err / scale).max())


CASES = [
    ("gmm_f64_p4096_s16", lambda: gen.gmm(1 << 22, seed=4), 4096, 16),
    ("uniform_i32_p1024", lambda: gen.uniform(1 << 22, 1024, 1), 1024, 0),
    ("zipf_i32_p256", lambda: gen.zipf(1 << 21, seed=2), 256, 0),
    ("f32_p64", lambda: gen.gmm(300_001, seed=9).astype(np.float32), 64, 0),
]


@pytest.mark.parametrize("name,make,p,s", CASES, ids=[c[0] for c in CASES])
def test_learned_sort_is_exact(name, make, p, s):
    keys = make()
    vals = np.arange(keys.shape[0], dtype=np.uint32)
    ref = oracle.sort(keys, p, s, 0, oracle.RANDOM, 8, vals=vals, want_bucket_of=True)
    gpu = run_gpu(keys, p, s, 0, oracle.RANDOM, 8, vals, classify=1)
    assert_same(gpu, ref)


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
def test_learned_with_regular_sampling(pairs):
    """Regular oversampling with the learned classifier: the network is
    trained on the regular sample and every key classified through it (the
    classification route); output, sizes and per-key buckets as the oracle's."""
    keys = gen.gmm(1 << 20, seed=11).astype(np.float32)
    vals = np.arange(keys.shape[0], dtype=np.uint32) if pairs else None
    ref = oracle.sort(keys, 64, 0, 0, oracle.REGULAR, 0, vals=vals, want_bucket_of=True)
    gpu = run_gpu(keys, 64, 0, 0, oracle.REGULAR, 0, vals, classify=1)
    assert_same(gpu, ref)


def test_training_lowers_the_loss_and_the_index_finds_most_buckets():
    """Training moves every layer and keeps the lowest loss (never above the
    spline start's); the index over the network's output holds most keys'
    buckets (a misprediction is a key outside its cell's splitter range), so
    a key costs a few splitter comparisons, far fewer than a binary search
    over all P - 1 splitters."""
    n, p = 1 << 22, 4096
    keys = gen.gmm(n, seed=4)
    gpu = run_gpu(keys, p, 16, 0, oracle.RANDOM, 8, classify=1, debug=False)
    st = gpu.stats
    assert st.status == 0
    first, last = gpu.mlp_loss
    assert last <= first
    P = gpu.plan.vbuckets
    steps_per_key = st.correction_steps / n
    assert st.mispredicted / n < 0.25
    assert steps_per_key < 0.5 * math.log2(P)
    print(f"loss {first:.3e} -> {last:.3e}; mispredicted {st.mispredicted / n:.4f}; "
          f"comparisons/key {steps_per_key:.2f} vs log2(P) = {math.log2(P):.1f}")
