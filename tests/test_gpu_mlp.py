"""GPU warm-start network (tcgen05 BF16 tensor-core layers, FP32 accumulation) against
the oracle's FP64 network, on random weights and standardised features spanning several
128-row tiles and a ragged tail."""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import sph

from gpu_util import gpu_ctx  # noqa: F401  (builds the library)

pytestmark = pytest.mark.gpu


def _params(rng, scale=0.4):
    p = np.zeros(sph.MLP_PARAMS)
    p[:sph.MLP_WEIGHTS] = rng.normal(scale=scale, size=sph.MLP_WEIGHTS)
    p[sph.MLP_WEIGHTS + 4: sph.MLP_WEIGHTS + 8] = 1.0       # feature std
    p[-1] = 1.0                                             # label std
    return p


def _bf16(x):
    """Round to bfloat16 (nearest even) and back, in float64."""
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _bf16_reference(p, f):
    """The same network with BF16-rounded layer operands (FP64 accumulation)."""
    from scipy.special import erf
    H = 64
    W1 = p[:256].reshape(H, 4); b1 = p[256:320]; W2 = p[320:320 + 4096].reshape(H, H)
    b2 = p[4416:4480]; W3 = p[4480:4544]; b3 = p[4544]
    g = lambda z: 0.5 * z * (1 + erf(z / np.sqrt(2)))
    a1 = g(_bf16(f) @ _bf16(W1).T + b1)
    a2 = g(_bf16(a1) @ _bf16(W2).T + b2)
    return a2 @ W3 + b3


@pytest.mark.parametrize("n", [1000, 128, 77, 200_003])
def test_forward_matches_oracle(n):
    import torch
    rng = np.random.default_rng(n)
    p = _params(rng)
    f = rng.normal(size=(n, 4))
    dp = torch.tensor(p, dtype=torch.float32, device="cuda")
    df = torch.tensor(f, dtype=torch.float32, device="cuda")
    y = torch.full((n,), np.nan, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert sph.sph_mlp_forward(dp, df, n, y, err) == sph.SPH_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    yg = y.cpu().numpy().astype(np.float64)
    ref = oracle.mlp_forward(p.astype(np.float32).astype(np.float64), f.astype(np.float32))
    # BF16 operands: normwise 2e-2 of the FP64 network
    assert np.linalg.norm(yg - ref) <= 2e-2 * np.linalg.norm(ref)
    # and 1e-3 of the same network with BF16-rounded operands (catches layout errors)
    emu = _bf16_reference(p.astype(np.float32).astype(np.float64), f.astype(np.float32))
    np.testing.assert_allclose(yg, emu, rtol=0, atol=1e-3 * np.abs(emu).max())


def test_gradient_matches_oracle():
    import torch
    rng = np.random.default_rng(11)
    n = 1000
    p = _params(rng, 0.3)
    f = rng.normal(size=(n, 4)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    dev = lambda a, dt=torch.float32: torch.tensor(a, dtype=dt, device="cuda")
    g = torch.zeros(sph.MLP_WEIGHTS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert sph.sph_mlp_grad(dev(p), dev(f), dev(t), n, g, loss, err) == sph.SPH_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    p64 = p.astype(np.float32).astype(np.float64)
    ref_loss, ref_g = oracle.mlp_loss_grad(p64, f.astype(np.float64), t.astype(np.float64))
    assert float(loss.item()) / n == pytest.approx(ref_loss, rel=2e-2)
    gg = g.cpu().numpy().astype(np.float64)
    # BF16 operands: normwise 2e-2 overall and per parameter group
    assert np.linalg.norm(gg - ref_g) <= 2e-2 * np.linalg.norm(ref_g)
    for lo, hi in [(0, 256), (256, 320), (320, 4416), (4416, 4480), (4480, 4544), (4544, 4545)]:
        assert np.linalg.norm(gg[lo:hi] - ref_g[lo:hi]) <= 5e-2 * np.linalg.norm(ref_g[lo:hi]) + 1e-7


def test_training_fits():
    import torch
    rng = np.random.default_rng(12)
    n = 4096
    f = rng.normal(size=(n, 4)).astype(np.float32) * np.array([1.0, 3.0, 0.5, 2.0], np.float32) + 1.0
    t = (np.sin(f[:, 0]) + 0.3 * f[:, 1] * f[:, 2] - 0.2 * f[:, 3]).astype(np.float32)
    p = _params(rng, 0.2)
    dp = torch.tensor(p, dtype=torch.float32, device="cuda")
    adam = torch.zeros(2 * sph.MLP_WEIGHTS, dtype=torch.float32, device="cuda")
    epochs = 60
    hist = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = sph.sph_mlp_train(torch.tensor(f, device="cuda"), torch.tensor(t, device="cuda"), n, dp, adam,
                           epochs, 256, 3e-3, 7, hist, err)
    assert st == sph.SPH_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    h = hist.cpu().numpy()
    assert h[-1] < 0.05 * h[0] and h[-1] < 0.05
    # the standardisation statistics went into the parameter block
    pp = dp.cpu().numpy()
    np.testing.assert_allclose(pp[sph.MLP_WEIGHTS:sph.MLP_WEIGHTS + 4], f.mean(0), rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(pp[sph.MLP_WEIGHTS + 4:sph.MLP_WEIGHTS + 8], f.std(0), rtol=1e-3)
    # the trained network predicts the training targets (oracle forward on its weights)
    fs = (f - pp[sph.MLP_WEIGHTS:sph.MLP_WEIGHTS + 4]) / pp[sph.MLP_WEIGHTS + 4:sph.MLP_WEIGHTS + 8]
    y = oracle.mlp_forward(pp.astype(np.float64), fs.astype(np.float64)) * pp[-1] + pp[-2]
    assert np.mean((y - t) ** 2) < 0.1 * np.var(t)
