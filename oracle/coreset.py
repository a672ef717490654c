"""Feature-based coreset and its epoch shuffle (Section 3.1; oracle, test infrastructure only).

The training coreset is the union over key frames t_k of the dilated feature d_k, each vertex a
4D training sample (x, y, z, t_k) labelled with the volume value there.  Samples are listed in
key-frame order, then in (z, y, x) order inside the Feature Bounding Box.  A sample's input
coordinates are FBB-normalised in float32: u_a = (a - lo_a) / (S_a - 1) for a in x, y, z (0 when
S_a == 1), and u_t = t / (T - 1) (0 when T == 1).

Training runs in epochs: epoch e visits every coreset sample once, in the order of a keyed
permutation pi_e of [0, N), batch b taking positions b*B .. b*B + B - 1.  pi_e is a 4-round
balanced Feistel network on k-bit integers (Luby and Rackoff) with cycle walking onto [0, N)
(Black and Rogaway, "Ciphers with Arbitrary Finite Domains", 2002):
* k = max(2, ceil(log2 N)) rounded up to even, h = k / 2;
* round keys K_r = output r of SplitMix64 seeded with key_e, where key_e is value e of stream 400
  of the seed (the library's SplitMix64 streams, oracle/rng.py);
* a round maps (L, R) to (R, L xor (mix(R xor K_r) mod 2^h)), mix being SplitMix64's output
  function;
* pi_e(x) applies the network to x = L * 2^h + R, then again while the result is >= N.
"""
import numpy as np

from . import index, rng


def build(mask, volume, key_frames):
    """Coreset of Section 3.1: (entries int64 [N][4] as (x, y, z, t), labels float32 [N], lo, size)."""
    d = index.dilate(mask)
    lo, size = index.fbb(d)
    ents, labels = [], []
    for t in key_frames:
        box = d[t, lo[2]:lo[2] + size[2], lo[1]:lo[1] + size[1], lo[0]:lo[0] + size[0]]
        z, y, x = np.nonzero(box)
        x, y, z = x + lo[0], y + lo[1], z + lo[2]
        ents.append(np.stack([x, y, z, np.full_like(x, t)], 1).astype(np.int64))
        labels.append(np.asarray(volume, np.float32)[t, z, y, x])
    ents = np.concatenate(ents) if ents else np.zeros((0, 4), np.int64)
    labels = np.concatenate(labels) if labels else np.zeros(0, np.float32)
    return ents, labels, lo, size


def coords_of(ents, lo, size, nt):
    """FBB-normalised float32 coordinates [N][4] of coreset samples (float32 divisions)."""
    out = np.zeros((ents.shape[0], 4), np.float32)
    for a in range(3):
        if size[a] > 1:
            out[:, a] = (ents[:, a] - lo[a]).astype(np.float32) / np.float32(size[a] - 1)
    if nt > 1:
        out[:, 3] = ents[:, 3].astype(np.float32) / np.float32(nt - 1)
    return out


def _mix(z):
    z = np.asarray(z, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * rng.M1
        z = (z ^ (z >> np.uint64(27))) * rng.M2
    return z ^ (z >> np.uint64(31))


def _bits(N):
    k = max(2, int(np.ceil(np.log2(max(N, 1)))))
    return k + (k & 1)


def permute(seed, epoch, N, x):
    """pi_epoch(x) for an array x of positions in [0, N)."""
    h = _bits(N) // 2
    mask = np.uint64((1 << h) - 1)
    key = rng.at(rng.at(seed, 400), epoch)
    K = [rng.at(key, r) for r in range(4)]

    def net(v):
        L, R = v >> np.uint64(h), v & mask
        for r in range(4):
            L, R = R, L ^ (_mix(R ^ K[r]) & mask)
        return (L << np.uint64(h)) | R

    y = net(np.asarray(x, np.uint64))
    while True:
        out = y >= np.uint64(N)
        if not out.any():
            return y.astype(np.int64)
        y[out] = net(y[out])


def batch(ents, labels, lo, size, nt, seed, epoch, b, B):
    """Coordinates [n][4] and targets [n] of batch b of epoch `epoch` (n = B, or less at the end)."""
    N = ents.shape[0]
    pos = np.arange(b * B, min(N, (b + 1) * B), dtype=np.int64)
    j = permute(seed, epoch, N, pos)
    return coords_of(ents[j], lo, size, nt), labels[j]
