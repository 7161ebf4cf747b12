"""Weight files (the model's checkpoint format) on the host: a round trip
keeps every member's arrays bit for bit, and malformed files are refused.
The same files through a GPU context, and NVE checkpoints, are in
tests/test_gpu_checkpoint.py."""
import numpy as np
import pytest

from paper_2604_21441_b300 import read_weights, write_weights


def _members(M, S, D, seed):
    rng = np.random.default_rng(seed)
    w = (D, 160, 128, 96, 1)
    return [[[(rng.standard_normal((w[l], w[l + 1])).astype(np.float32),
               rng.standard_normal(w[l + 1]).astype(np.float32)) for l in range(4)]
             for _ in range(S)] for _ in range(M)]


def test_round_trip(tmp_path):
    zs = (1, 6, 8)
    mem = _members(2, 3, 240, 5)
    path = str(tmp_path / "model.npz")
    write_weights(path, zs, mem)
    zs2, mem2 = read_weights(path)
    assert zs2 == zs and len(mem2) == 2
    for a, b in zip(mem, mem2):
        for la, lb in zip(a, b):
            assert len(la) == len(lb) == 4
            for (Wa, ba), (Wb, bb) in zip(la, lb):
                assert Wb.dtype == np.float32 and Wa.shape == Wb.shape
                assert np.array_equal(Wa, Wb) and np.array_equal(ba, bb)


def test_refusals(tmp_path):
    zs = (1, 8)
    mem = _members(1, 2, 128, 6)
    with pytest.raises(ValueError):  # a member with the wrong species count
        write_weights(str(tmp_path / "a.npz"), zs, [mem[0][:1]])
    path = str(tmp_path / "b.npz")
    write_weights(path, zs, mem)
    with np.load(path) as f:
        arrays = dict(f)
    arrays["format"] = np.int64(99)
    np.savez(str(tmp_path / "c.npz"), **arrays)
    with pytest.raises(ValueError):  # unknown format
        read_weights(str(tmp_path / "c.npz"))
    arrays["format"] = np.int64(1)
    for k in [k for k in arrays if k.startswith("m0_s1_")]:
        del arrays[k]
    np.savez(str(tmp_path / "d.npz"), **arrays)
    with pytest.raises(ValueError):  # a species without layers
        read_weights(str(tmp_path / "d.npz"))
