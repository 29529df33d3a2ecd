"""The warm-start network's CUDA kernels (BF16 tensor-core products, FP32
accumulation) against the FP64 oracle of oracle/mlp.py, which applies the same
BF16 roundings: outputs, loss, every gradient block, and an Adam step."""
import numpy as np
import pytest

from oracle import mlp as om

pytestmark = pytest.mark.gpu


def _setup(sizes, B, seed):
    import torch
    from paper_1702_01335_gb300.warmstart import Mlp
    rng = np.random.default_rng(seed)
    p = om.init_params(rng, sizes)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    flat = np.concatenate([np.concatenate([p["W%d" % i].ravel(), p["b%d" % i]]) for i in (1, 2, 3)])
    flat = flat.astype(np.float32)
    net = Mlp(sizes, max_batch=max(B, 64))
    net.set_params(flat)
    pf = net.unpack(flat.astype(np.float64))  # the float32 masters, as the oracle's parameters
    x = rng.standard_normal((B, sizes[0])).astype(np.float32)
    t = rng.standard_normal((B, sizes[-1])).astype(np.float32)
    xd, td = (torch.tensor(a, device="cuda") for a in (x, t))
    return net, pf, x.astype(np.float64), t.astype(np.float64), xd, td


U_BF16 = 2.0 ** -8   # the largest rounding error of a BF16 value, relative (8 significant bits)
KAPPA = 2.0          # rounding differences an entry can inherit, one BF16 level each


def error_bounds(p, x, t):
    """Per-entry bounds on |GPU - oracle|: KAPPA U_BF16 times the magnitude of the
    terms the entry accumulates, sum_k |a_k| |b_k| over the BF16 operands of its
    product (the oracle's).  The two sides round the same weights to the same BF16
    values; they differ where an activation or an incoming gradient, whose unrounded
    values are a few FP32 ulps apart, lies next to a BF16 rounding boundary and rounds
    to the neighbouring value on one side (a change of at most U_BF16 relative), and by
    the FP32 accumulation (K 2^-24 relative, far below).  A flipped operand changes
    the entry by at most U_BF16 times its own term; KAPPA allows for the operand's own
    flip and for the smaller change it inherits from flips one layer up."""
    A = np.abs
    y, (_, z1, h1, z2, h2) = om.forward(p, x)
    B, M = y.shape
    W1, W2, W3 = (om.bf16(p[k]) for k in ("W1", "W2", "W3"))
    bx, bh1, bh2 = om.bf16(x), om.bf16(h1), om.bf16(h2)
    dy = 2.0 * (y - t) / (B * M)
    bdy = om.bf16(dy)
    dz2 = (bdy @ W3) * om.gelu_grad(z2)
    bdz2 = om.bf16(dz2)
    dz1 = (bdz2 @ W2) * om.gelu_grad(z1)
    bdz1 = om.bf16(dz1)
    m = {"y": A(bh2) @ A(W3).T + A(p["b3"]),
         "W3": A(bdy).T @ A(bh2), "b3": A(dy).sum(0),
         "W2": A(bdz2).T @ A(bh1), "b2": A(dz2).sum(0),
         "W1": A(bdz1).T @ A(bx), "b1": A(dz1).sum(0)}
    return {k: KAPPA * U_BF16 * v for k, v in m.items()}


def _within(got, ref, bound):
    return bool(np.all(np.abs(got - ref) <= bound))


@pytest.mark.parametrize("sizes,B", [((6, 32, 32, 40), 37), ((6, 256, 256, 512), 256)])
def test_forward_loss_and_gradients_match_oracle(sizes, B):
    """Element by element: every output and every gradient entry lies within its own
    bound (error_bounds); the loss within 1e-4 relative."""
    net, pf, x, t, xd, td = _setup(sizes, B, seed=3)
    E = error_bounds(pf, x, t)
    y_gpu = net.forward(xd).cpu().numpy()
    y_ora, _ = om.forward(pf, x)
    assert _within(y_gpu, y_ora, E["y"]), np.max(np.abs(y_gpu - y_ora) / E["y"])
    loss, g = net.loss_grad(xd, td, want_grad=True)
    L_ora, g_ora = om.loss_and_grads(pf, x, t)
    assert abs(loss / L_ora - 1) < 1e-4
    gg = net.unpack(g.astype(np.float64))
    ratios = {}
    for k in g_ora:
        ratios[k] = float(np.max(np.abs(gg[k] - g_ora[k]) / E[k]))
        assert _within(gg[k], g_ora[k], E[k]), (k, ratios[k])
        # the bounds are tight enough to matter: relative to the entries they bound
        # they stay well below 1
        rel = E[k] / np.maximum(np.abs(g_ora[k]), 1e-30)
        assert np.median(rel) < 0.3, (k, float(np.median(rel)))
    print("\n[mlp %s, B=%d] max |gpu - oracle| / bound: %s" % (
        sizes, B, ", ".join("%s %.2f" % kv for kv in sorted(ratios.items()))))
    net.close()


def test_adam_step_matches_oracle():
    net, pf, x, t, xd, td = _setup((6, 32, 32, 40), 37, seed=4)
    _, g = net.loss_grad(xd, td, want_grad=True)
    net.adam(1e-3)
    after = net.unpack(net.get_params().astype(np.float64))
    ref = {k: v.copy() for k, v in pf.items()}
    om.adam_step(ref, net.unpack(g.astype(np.float64)), {}, lr=1e-3)
    for k in ref:
        assert np.allclose(after[k], ref[k], rtol=0, atol=1e-6), k
    net.close()


def test_training_fits_a_smooth_map():
    """A few hundred Adam steps fit a smooth 6 -> 40 map (the loss drops 20-fold)."""
    import torch
    from paper_1702_01335_gb300.warmstart import Mlp
    rng = np.random.default_rng(5)
    A = rng.standard_normal((6, 40)) * 0.5
    x = rng.standard_normal((512, 6))
    t = np.sin(x @ A)
    net = Mlp((6, 64, 64, 40), max_batch=512, seed=1)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    first, _ = net.loss_grad(xd, td)
    for _ in range(400):
        loss, _ = net.loss_grad(xd, td)
        net.adam(3e-3)
    assert loss < first / 20, (first, loss)
    net.close()
