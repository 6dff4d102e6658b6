"""Seeded input generators: Philox4x32-10 against the published known-answer
vectors (Salmon et al., SC'11, Random123 distribution) and SU(3) links."""
import numpy as np

import synth


def test_philox_known_answers():
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = synth.philox4x32_10(*ctr, *key)
        assert tuple(int(g) for g in got) == want


def test_gauge_links_are_su3_and_reproducible():
    U = synth.gauge_field((4, 4, 2, 2), 0.3, 7)
    u = U.reshape(-1, 3, 3)
    assert np.abs(np.einsum("lij,lkj->lik", u, u.conj()) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    # distance from the identity scales with eps
    d = np.abs(u - np.eye(3)).mean()
    assert 0.02 < d < 0.3
    assert np.array_equal(U, synth.gauge_field((4, 4, 2, 2), 0.3, 7))
    assert not np.array_equal(U, synth.gauge_field((4, 4, 2, 2), 0.3, 8))


def test_uniform_vectors_exact_dyadic():
    W = synth.uniform_vectors((2, 2, 2, 4), 3, 11)
    assert W.shape == (3, 4, 2, 2, 2, 4, 3)
    for part in (W.real, W.imag):
        assert part.min() >= -1 and part.max() < 1
        assert np.all(part * 2.0 ** 31 == np.round(part * 2.0 ** 31))
    # component 2q+1 of site s in vector j comes from words 2, 3 of block (s, q, j)
    r = synth.philox4x32_10(5, 2, 1, synth.TAG_TESTVEC, 11, 0)
    v = W[1].reshape(-1, 12)[5, 5]
    assert v.real == np.int32(np.uint32(r[2])) * 2.0 ** -31
    assert v.imag == np.int32(np.uint32(r[3])) * 2.0 ** -31


def test_z2_noise():
    eta = synth.z2_noise((2, 2, 2, 2), 2, 3)
    assert np.allclose(np.abs(eta), 1.0)
    assert set(np.unique(np.sign(eta.real))) == {-1.0, 1.0}
