"""The seeded input generators: Philox4x32-10 known-answer vectors and the stated matrix structure."""
import numpy as np

import synth


def test_philox_known_answers():
    # known-answer vectors published with the Random123 distribution (Salmon et al., SC'11)
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = synth.philox4x32_10(np.array([ctr], dtype=np.uint32), key)[0]
        assert tuple(int(v) for v in got) == want


def test_random_u32_offsets_are_consistent():
    full = synth.random_u32(5, 2, 103)
    for off, cnt in [(0, 1), (1, 7), (13, 50), (99, 4)]:
        np.testing.assert_array_equal(synth.random_u32(5, 2, cnt, offset=off), full[off:off + cnt])


def test_dominant_system_structure():
    n, f = 300, 1.05
    A, B, Xs = synth.dominant_system(n, f, seed=1, nrhs=2)
    M = np.abs(A)
    np.fill_diagonal(M, 0.0)
    off = M.sum(axis=1)                                                # exact: integers times 2**-31
    np.testing.assert_array_equal(np.abs(np.diag(A)), f * off)
    assert np.all(np.abs(A - np.diag(np.diag(A))) <= 1.0)
    assert (np.diag(A) < 0).any() and (np.diag(A) > 0).any()           # random signs
    np.testing.assert_array_equal(B, A @ Xs)
    assert np.all(np.abs(Xs) <= 1.0)
    A2, _, _ = synth.dominant_system(n, f, seed=1, nrhs=2)
    np.testing.assert_array_equal(A, A2)


def test_hard_system_structure():
    A, _, _ = synth.hard_system(64, 1.25, seed=3)
    off = A - np.diag(np.diag(A))
    assert np.all(off >= 0) and np.all(off < 1)
    np.testing.assert_array_equal(np.diag(A), 1.25 * off.sum(axis=1))


def test_batch_shapes_ranges():
    n, f = synth.batch_shapes(4096, 64, 1024, 1.05, 2.0, seed=2)
    assert n.min() >= 64 and n.max() <= 1024
    assert f.min() >= 1.05 and f.max() <= 2.0
    # log-uniform: the median is near the geometric mean sqrt(64 * 1025) ~ 256
    assert 220 < np.median(n) < 300


def test_symmetric_generator_structure():
    A, B, Xs = synth.symmetric_system(40, 1.2, seed=9, nrhs=2)
    np.testing.assert_array_equal(A, A.T)
    d = np.abs(np.diag(A))
    off = np.abs(A).sum(axis=1) - d
    np.testing.assert_allclose(off / d, 1 / 1.2, rtol=1e-15)
    np.testing.assert_allclose(B, A @ Xs, rtol=0, atol=0)
