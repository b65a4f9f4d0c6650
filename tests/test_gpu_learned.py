"""The learned classifier on the GPU (params.classify = BSPS_LEARNED).

* loss and gradient of the GPU kernels vs the float64 CPU oracle (oracle/mlp.py),
  relative error <= 1e-3 (FP32 accumulation over <= 16384 points);
* sorts with the learned classifier are bit-identical to the oracle (keys,
  payloads, bucket sizes, splitters, per-key buckets): the correction makes the
  bucket exact whatever the network predicts;
* what training gains: the trained network's predictions need fewer correction
  steps than a binary search over all splitters, and its loss drops.
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


def test_training_gains_over_the_plain_search():
    n, p = 1 << 22, 4096
    keys = gen.gmm(n, seed=4)
    gpu = run_gpu(keys, p, 16, 0, oracle.RANDOM, 8, classify=1, debug=False)
    st = gpu.stats
    assert st.status == 0
    first, last = gpu.mlp_loss
    assert last < first                       # training lowered the loss
    P = gpu.plan.vbuckets
    steps_per_key = st.correction_steps / n
    # a plain binary search over the P-1 splitters takes ~log2(P) comparisons
    assert steps_per_key < math.log2(P)
    print(f"loss {first:.3e} -> {last:.3e}; mispredicted {st.mispredicted / n:.3f}; "
          f"correction steps/key {steps_per_key:.2f} vs log2(P) = {math.log2(P):.1f}")
