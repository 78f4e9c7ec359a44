"""The seeded generator gives the same bytes through numpy and through torch."""
import numpy as np

import synth


def test_numpy_and_torch_agree():
    for seed, stream, n in [(0, 0, 0), (0, 0, 1), (1, 2, 37), (3, 0, 4096 + 3), (7, 4, 100_001)]:
        a = synth.bytes_np(seed, stream, n)
        b = synth.bytes_torch(seed, stream, n, chunk_words=1000).numpy()
        assert a.dtype == np.uint8 and a.size == n
        assert np.array_equal(a, b)


def test_splitmix64_first_output_matches_published_definition():
    # Straight scalar transcription of SplitMix64's step, seeded at base.
    mask = (1 << 64) - 1
    base = (5 << 40) + (2 << 32)
    x = (base + 0x9E3779B97F4A7C15) & mask
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    z = z ^ (z >> 31)
    assert int(synth.words_np(5, 2, 1)[0]) == z


def test_streams_differ_and_iv_layout():
    assert not np.array_equal(synth.bytes_np(0, 0, 64), synth.bytes_np(0, 1, 64))
    iv = synth.iv_bytes(3, counter0=0x01020304)
    assert iv.tolist()[12:] == [1, 2, 3, 4]
    assert synth.key_bytes(3, 192).size == 24
    u = synth.uniform01(1, synth.STREAM_LENGTH, 10000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.02
