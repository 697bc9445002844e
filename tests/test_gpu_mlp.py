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


@pytest.mark.parametrize("n", [1000, 128, 77])
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
