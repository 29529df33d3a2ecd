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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("sizes,B", [((6, 32, 32, 40), 37), ((6, 256, 256, 512), 256)])
def test_forward_loss_and_gradients_match_oracle(sizes, B):
    net, pf, x, t, xd, td = _setup(sizes, B, seed=3)
    y_gpu = net.forward(xd).cpu().numpy()
    y_ora, _ = om.forward(pf, x)
    assert _rel(y_gpu, y_ora) < 1e-4
    loss, g = net.loss_grad(xd, td, want_grad=True)
    L_ora, g_ora = om.loss_and_grads(pf, x, t)
    assert abs(loss / L_ora - 1) < 1e-4
    gg = net.unpack(g.astype(np.float64))
    for k in g_ora:
        assert _rel(gg[k], g_ora[k]) < 2e-3, (k, _rel(gg[k], g_ora[k]))
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
