"""The torch pair digest of the full-size tests equals the oracle's hash and
a numpy degree count (CPU tensors; no GPU)."""
import numpy as np
import pytest

from gpu_digest import Digest
from oracle import oracle as orc


def test_torch_digest_equals_oracle_hash_and_bincount():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    n = 5000
    # ids over the full 32-bit range as well as small ones, so that the sign
    # bit of i << 32 and of every product is exercised
    i = np.concatenate([rng.integers(0, n, 20000), rng.integers(0, n, 50)]).astype(np.uint32)
    j = np.concatenate([rng.integers(0, 2**32, 20000), rng.integers(0, n, 50)]).astype(np.uint32)
    keys = (i.astype(np.uint64) << np.uint64(32)) | j.astype(np.uint64)
    pairs = torch.from_numpy(np.stack([i, j], axis=1).view(np.int32))
    dg = Digest(n, "cpu")
    dg.add(pairs[:7000], block=3000)
    dg.add(pairs[7000:])
    assert dg.count == keys.size
    assert dg.hash == orc.pair_hash(keys)
    want = sum(orc.mix64(int(k)) for k in keys[:200]) % (1 << 64)
    small = Digest(n, "cpu")
    small.add(pairs[:200])
    assert small.hash == want
    assert np.array_equal(dg.degree.numpy(), np.bincount(i, minlength=n))
