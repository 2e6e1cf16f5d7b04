"""The warm-start network on the GPU against the CPU oracle of the same network: forward
output and gradients (BF16 weights, FP32 accumulation, so the oracle runs in FP64 with the
same BF16-rounded weights), and one Adam step."""
import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _split(flat):
    shapes = [(32, 3, 3, 3), (32,), (32, 32, 3, 3), (32,), (32, 32, 3, 3), (32,), (2, 32, 3, 3), (2,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(flat[o:o + n].reshape(s))
        o += n
    return out


@pytest.mark.parametrize("B,H,W,dil", [(2, 18, 21, (1, 1, 1, 1)), (1, 35, 33, (1, 2, 4, 8)), (2, 20, 19, (2, 4, 8, 1))])
def test_forward_and_gradients_match_oracle(B, H, W, dil, monkeypatch):
    # the FP32-activation path (training's forward); the tensor-core forward is tested below
    monkeypatch.setenv("IGAMG_NN_TC", "0")
    torch = _torch()
    from paper_1705_09282_gb300.warmstart import Network
    net = Network(seed=5, dilations=dil)
    flat = net.get_params()
    rng = np.random.default_rng(3)
    x = rng.standard_normal((B, 3, H, W)).astype(np.float32)
    t = rng.standard_normal((B, 2, H, W)).astype(np.float32)
    xg, tg = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    out = net.forward(xg).cpu().numpy()
    params = _split(flat.astype(np.float64))
    for k in (0, 2, 4, 6):                       # weights as the GPU uses them (BF16)
        params[k] = _bf16(params[k])
    ref = cnn.CNN(params, dil)
    mask = np.zeros((2, H, W))
    mask[0, 1:-1, 1:-1] = 1.0
    mask[1, :-1, :-1] = 1.0
    o_ref = ref.forward(x.astype(np.float64), np.ones((2, H, W)))
    assert np.abs(out - o_ref).max() <= 2e-4 * np.abs(o_ref).max()
    loss, grad = net.loss_grad(xg, tg)
    loss_ref, g_ref = ref.loss_and_grads(x.astype(np.float64), mask, t.astype(np.float64) * mask[None])
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    g_ref_flat = np.concatenate([g.ravel() for g in g_ref])
    assert np.abs(grad - g_ref_flat).max() <= 1e-3 * np.abs(g_ref_flat).max()


def test_training_reduces_loss_and_adam_matches_oracle():
    torch = _torch()
    from paper_1705_09282_gb300.warmstart import Network
    net = Network(seed=9)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 20, 20)).astype(np.float32)
    t = np.stack([np.tanh(x[:, 0] + 0.5 * x[:, 1]), np.tanh(x[:, 1] - x[:, 2])], axis=1).astype(np.float32)
    xg, tg = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    p0 = net.get_params().astype(np.float64)
    _, g0 = net.loss_grad(xg, tg)
    l_first = net.train_step(xg, tg, lr=1e-3)
    p1 = net.get_params().astype(np.float64)
    # first Adam step: w -= lr * g / (|g| + eps)
    want = p0 - 1e-3 * g0 / (np.abs(g0) + 1e-8)
    assert np.abs(p1 - want).max() <= 1e-6
    for _ in range(60):
        l_last = net.train_step(xg, tg, lr=3e-3)
    assert l_last < 0.5 * l_first


@pytest.mark.parametrize("B,H,W,dil", [(2, 18, 21, (1, 1, 1, 1)), (1, 35, 33, (1, 2, 4, 8)), (3, 67, 66, (1, 2, 4, 8)),
                                       (1, 131, 130, (2, 4, 8, 1))])
def test_tensor_core_forward_matches_bf16_reference(B, H, W, dil):
    # inference runs the two 32 -> 32 layers as tcgen05 implicit GEMMs: BF16 weights and BF16
    # activations, FP32 accumulation in tensor memory.  Reference: the oracle's layers in FP64
    # with those layers' inputs rounded to BF16 (images of several 128-pixel tiles with a
    # ragged last tile, every dilation)
    torch = _torch()
    from paper_1705_09282_gb300.warmstart import Network
    net = Network(seed=7, dilations=dil)
    params = _split(net.get_params().astype(np.float64))
    for k in (0, 2, 4, 6):
        params[k] = _bf16(params[k])
    rng = np.random.default_rng(11)
    x = rng.standard_normal((B, 3, H, W)).astype(np.float32)
    out = net.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    a = cnn.gelu(cnn.conv3x3(x.astype(np.float64), params[0], params[1], dil[0]))
    a = cnn.gelu(cnn.conv3x3(_bf16(a), params[2], params[3], dil[1]))
    a = cnn.gelu(cnn.conv3x3(_bf16(a), params[4], params[5], dil[2]))
    ref = cnn.conv3x3(a, params[6], params[7], dil[3])
    assert np.abs(out - ref).max() <= 2e-3 * np.abs(ref).max(), np.abs(out - ref).max() / np.abs(ref).max()
