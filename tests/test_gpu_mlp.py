"""The tensor-core surrogate network against the FP64 CPU reference
(oracle/mlp.py): forward outputs, the loss and every parameter gradient,
element by element, within BF16 tolerances.

The bounds come from the arithmetic: the operands of every product are BF16
(8 significant bits, relative rounding 2^-9), the accumulators FP32.  A
forward output carries a few roundings of 2^-9 per layer; a gradient element
is a sum over the batch of products of a BF16 activation and a BF16 upstream
gradient, each off by ~1% after four layers, so an element is within 5% of
itself plus 1% of its tensor's largest element (the absolute part covers
sums that cancel)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1608_01125_gb300 import binding

pytestmark = pytest.mark.gpu


def _setup(m, seed):
    import __graft_entry__
    __graft_entry__.build()
    import torch
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((m, 24))
    y = rng.standard_normal(m) * 1.5 + 0.5
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    norm = np.concatenate([np.zeros(24), np.ones(24)])
    return p, x, y, dev(binding.mlp_flatten(p)), dev(norm), dev(x), dev(y)


@pytest.mark.parametrize("m", [1, 127, 128, 1000, 70001])
def test_forward_matches_fp64_reference(m):
    p, x, y, P, N, X, Y = _setup(m, 3)
    out = binding.mlp_forward(P, N, X).cpu().numpy()
    ref, _ = mlp.forward(p, x)
    # BF16 operands (8 significant bits) through 4 layers
    err = np.abs(out - ref)
    scale = np.abs(ref).mean() + 1e-3
    assert err.max() <= 0.08 * scale + 0.05 * np.abs(ref).max(), (err.max(), scale)
    assert np.median(err) <= 0.02 * scale


def test_normalisation_is_applied():
    import torch
    p, x, y, P, N, X, Y = _setup(500, 4)
    mean = np.linspace(-1, 1, 24)
    inv = np.linspace(0.5, 2, 24)
    raw = x / inv + mean
    N2 = torch.from_numpy(np.concatenate([mean, inv]).astype(np.float32)).cuda()
    a = binding.mlp_forward(P, N2, torch.from_numpy(raw.astype(np.float32)).cuda()).cpu().numpy()
    b = binding.mlp_forward(P, N, X).cpu().numpy()
    assert np.allclose(a, b, atol=0.05 * np.abs(b).max())


def _check_grads(gv, gref):
    for k, _ in binding.MLP_ORDER:
        a, r = gv[k].reshape(-1), gref[k].reshape(-1)
        top = np.abs(r).max()
        assert top > 0, k
        err = np.abs(a - r)
        bad = err > 0.05 * np.abs(r) + 0.01 * top
        assert not bad.any(), (k, int(bad.sum()), float(err.max() / top))
        rel = np.linalg.norm(a - r) / np.linalg.norm(r)
        assert rel < 0.02, (k, rel)


# 1 and 130 rows: one partial 128-row tile; 4096: eight full 512-row blocks;
# 5077: a ragged last block and a ragged last tile
@pytest.mark.parametrize("m", [1, 130, 4096, 5077])
def test_gradients_match_fp64_reference(m):
    p, x, y, P, N, X, Y = _setup(m, 5)
    g, loss = binding.mlp_grad(P, N, X, Y)
    L, gref = mlp.loss_and_grads(p, x, y)
    assert abs(float(loss.item()) / m - L) <= 0.03 * abs(L) + 1e-3
    _check_grads(binding.mlp_unflatten(g.cpu().numpy().astype(np.float64)), gref)


def test_gradients_add_over_batch_splits():
    """The mean gradient of m rows is the row-weighted mean of the gradients
    of two parts (split at 700, inside a block and inside a tile); only the
    BF16 rounding of the 1/m-scaled upstream gradient and the FP32 summation
    order differ."""
    m, k = 3000, 700
    p, x, y, P, N, X, Y = _setup(m, 7)
    g = binding.mlp_grad(P, N, X, Y)[0].cpu().numpy().astype(np.float64)
    g1 = binding.mlp_grad(P, N, X[:k].contiguous(), Y[:k].contiguous())[0].cpu().numpy()
    g2 = binding.mlp_grad(P, N, X[k:].contiguous(), Y[k:].contiguous())[0].cpu().numpy()
    s = (k * g1.astype(np.float64) + (m - k) * g2.astype(np.float64)) / m
    gv, sv = binding.mlp_unflatten(g), binding.mlp_unflatten(s)
    for name, _ in binding.MLP_ORDER:
        a, r = gv[name].reshape(-1), sv[name].reshape(-1)
        assert np.all(np.abs(a - r) <= 0.01 * np.abs(r) + 0.005 * np.abs(r).max()), name


def test_surrogate_objective_gradients_match_fp64_reference():
    import torch
    m = 4096
    p, x, y, P, N, X, Y = _setup(m, 6)
    rng = np.random.default_rng(8)
    lab = rng.gamma(1.5, 4.0, m) * (rng.random(m) < 0.7)  # many zero labels
    st = rng.gamma(2.0, 2.0, m)
    scale = 1.3
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    g, loss = binding.mlp_grad(P, N, X, dev(lab), kind=1, baseline=dev(st), scale=scale)
    out, cache = mlp.forward(p, x)
    B = scale * st
    L = mlp.loss_mean(out, lab, B)
    gref = mlp.backward(p, cache, mlp.loss_mean_grad(out, lab, B))
    assert abs(float(loss.item()) / m - L) <= 0.03 * abs(L) + 1e-3
    _check_grads(binding.mlp_unflatten(g.cpu().numpy().astype(np.float64)), gref)


def test_gradients_are_reproducible_bit_for_bit():
    """The weight gradients are summed over the batch in a fixed order (per-block
    slices added in block order, no atomics), so two calls on the same inputs
    give the same bits, and so does training."""
    m = 5077
    p, x, y, P, N, X, Y = _setup(m, 9)
    g1, l1 = binding.mlp_grad(P, N, X, Y)
    g2, l2 = binding.mlp_grad(P, N, X, Y)
    assert np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())
