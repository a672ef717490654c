"""Pin of the oracle's bf16 rounding against torch's bf16 conversion (a library routine).  CPU only."""
import numpy as np
import torch

from oracle import precision


def test_bf16_round_matches_torch():
    r = np.random.default_rng(0)
    x = np.concatenate([r.standard_normal(100000).astype(np.float32) * 10.0 ** r.integers(-30, 30, 100000),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, 1e-40, np.inf, -np.inf], np.float32)])
    # exact ties: low 16 bits = 0x8000, both even and odd upper halves
    ties = (r.integers(0, 2 ** 15, 2000, dtype=np.uint32) << 16 | 0x8000).astype(np.uint32).view(np.float32)
    x = np.concatenate([x, ties[np.isfinite(ties)]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = precision.bf16_round(x)
    assert np.array_equal(got, ref)
