"""The random-gather diagnostic (fhash_diag_random_gather) gathers what it claims: its checksum equals
the sum of the table entries at the SplitMix64 positions, recomputed on the host (oracle/rng.py), for
each width; bad arguments are rejected before any launch."""
import numpy as np
import pytest

from oracle import rng

from _util import fh, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [4, 8, 16])
def test_random_gather_checksum(width):
    t = torch()
    table = t.rand(1 << 16, dtype=t.float32, device="cuda")
    out = t.zeros(1, dtype=t.float32, device="cuda")
    n, seed = 5003, 9
    fh().fhash_diag_random_gather(table, width, n, seed, out)
    t.cuda.synchronize()
    slots = table.numel() * 4 // width
    idx = (rng.at(seed, np.arange(n)) % np.uint64(slots)).astype(np.int64)
    ref = table.cpu().numpy().astype(np.float64).reshape(-1, width // 4)[idx].sum()
    assert abs(float(out.item()) - ref) <= 1e-4 * abs(ref)


def test_random_gather_rejects_bad_arguments():
    t = torch()
    table = t.rand(1024, dtype=t.float32, device="cuda")
    out = t.zeros(1, dtype=t.float32, device="cuda")
    with pytest.raises(fh().FHashError):
        fh().fhash_diag_random_gather(table, 12, 10, 1, out)  # width
    with pytest.raises(fh().FHashError):
        fh().fhash_diag_random_gather(table.cpu(), 4, 10, 1, out)  # host table
