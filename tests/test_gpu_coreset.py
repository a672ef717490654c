"""GPU parity of the feature-based coreset (Section 3.1) against the oracle, through the C ABI.

- fhash_coreset_build: the sample count equals the oracle's (dilated feature at the key frames), from
  a host and from a device volume.
- fhash_coreset_batch: coordinates and labels of first, middle and ragged last batches are bit-exact
  (integer and float32-division work on both sides) for two seeds and epochs; the batches of an
  epoch cover the coreset exactly once.
- fhash_coreset_train_step: the loss of the first step equals the oracle's on the same batch with the
  library's documented initial parameters, within 1e-5 relative; eight epochs at least halve it.
- Argument errors: no coreset, a batch past the end, key frames out of order.
"""
import numpy as np
import pytest

from synth import workloads
from oracle import coreset, rng, train

from _util import build, fh, to_dev, torch

pytestmark = pytest.mark.gpu
W = workloads.SMALL
KEYS = [0, 3, 7]
SEED = 7


@pytest.fixture(scope="module")
def small():
    f, m = workloads.make_field_and_mask(W)
    ents, labels, lo, size = coreset.build(m, f, KEYS)
    return dict(field=f, mask=m, ents=ents, labels=labels, lo=lo, size=size)


def _batch(model, seed, epoch, b, B, N):
    n = min(B, N - b * B)
    c = torch().empty((n, 4), dtype=torch().float32, device="cuda")
    t = torch().empty(n, dtype=torch().float32, device="cuda")
    got = fh().fhash_coreset_batch(model, seed, epoch, b, B, c, t)
    assert got == n
    return c.cpu().numpy(), t.cpu().numpy()


def test_coreset_build_and_batches(small):
    model = build(W, mask=small["mask"], seed=SEED)
    with pytest.raises(fh().FHashError):
        fh().fhash_coreset_batch(model, 1, 0, 0, 16, torch().empty((16, 4), device="cuda"),
                                 torch().empty(16, device="cuda"))
    N = fh().fhash_coreset_build(model, small["field"], KEYS)
    assert N == small["ents"].shape[0] > 0
    assert fh().fhash_coreset_build(model, to_dev(small["field"]), KEYS) == N  # device volume
    nt = W["dims"][3]
    B = 1000
    nbatch = (N + B - 1) // B
    for seed, epoch in ((1, 0), (99, 5)):
        for b in sorted({0, nbatch // 2, nbatch - 1}):
            c, t = _batch(model, seed, epoch, b, B, N)
            rc, rt = coreset.batch(small["ents"], small["labels"], small["lo"], small["size"], nt, seed, epoch, b, B)
            assert np.array_equal(c, rc) and np.array_equal(t, rt), (seed, epoch, b)
    # one epoch covers the coreset exactly once
    allc = np.concatenate([_batch(model, 3, 2, b, B, N)[0] for b in range(nbatch)])
    want = coreset.coords_of(small["ents"], small["lo"], small["size"], nt)
    assert np.array_equal(np.unique(allc, axis=0), np.unique(want, axis=0)) and allc.shape == want.shape
    with pytest.raises(fh().FHashError):
        _batch(model, 1, 0, nbatch, B, N + B)  # past the end
    with pytest.raises(fh().FHashError):
        fh().fhash_coreset_build(model, small["field"], [3, 0])
    fh().fhash_check(model)


def test_coreset_training(small):
    model = build(W, mask=small["mask"], seed=SEED)
    info = fh().fhash_get_info(model)
    N = fh().fhash_coreset_build(model, small["field"], KEYS)
    B = 4096
    hp = tuple(float(np.float32(x)) for x in W["adam"])
    # first step against the oracle, from the library's documented initial parameters
    rc, rt = coreset.batch(small["ents"], small["labels"], small["lo"], small["size"], W["dims"][3], 11, 0, 0, B)
    table = rng.InitTable(SEED, info["F"], float(np.float32(W["init_range"])))
    p = rng.init_mlp(SEED, info["mlp_dims"])
    L, _, _, _ = train.loss_and_grads(info["res"], info["base"], info["F"], info["mlp_dims"], table, p, rc, rt)
    loss = np.zeros(1, np.float64)
    fh().fhash_coreset_train_step(model, 11, 0, 0, B, hp, loss)
    assert abs(loss[0] - L) <= 1e-5 * L, (loss[0], L)
    first = loss[0]
    for epoch in range(8):
        for b in range((N + B - 1) // B):
            if epoch == 0 and b == 0:
                continue
            fh().fhash_coreset_train_step(model, 11, epoch, b, B, hp, loss)
    assert loss[0] < 0.5 * first, (first, loss[0])
    fh().fhash_check(model)


def test_coreset_without_mask_covers_every_voxel():
    # no mask: the feature is the whole volume, so the coreset is every voxel of every key frame
    dims = (9, 5, 7, 4)
    w = dict(W, dims=dims, schedule=dict(mode="explicit", res=[[3, 3, 3, 2], [9, 5, 7, 4]]))
    model = build(w, mask=None, dims=dims)
    vol = np.arange(np.prod(dims[::-1]), dtype=np.float32).reshape(dims[::-1])
    keys = [1, 3]
    N = fh().fhash_coreset_build(model, vol, keys)
    assert N == 9 * 5 * 7 * len(keys)
    c = torch().empty((N, 4), dtype=torch().float32, device="cuda")
    t = torch().empty(N, dtype=torch().float32, device="cuda")
    assert fh().fhash_coreset_batch(model, 5, 0, 0, N, c, t) == N
    m = np.ones(dims[::-1], np.uint8)
    ents, labels, lo, size = coreset.build(m, vol, keys)
    rc, rt = coreset.batch(ents, labels, lo, size, dims[3], 5, 0, 0, N)
    assert np.array_equal(c.cpu().numpy(), rc) and np.array_equal(t.cpu().numpy(), rt)
    assert np.array_equal(np.sort(t.cpu().numpy()), np.sort(vol[keys].ravel()))
