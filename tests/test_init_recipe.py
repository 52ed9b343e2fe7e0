"""The seeded "random" initial values (Algorithm 1, first step, which leaves the initial values
to the user): the host recipe in synth, pinned against the generator's published definition and
the recipe's own formulas. The CUDA library draws the same values on the device
(tests/test_gpu_init.py)."""
import numpy as np

import synth

MASK = (1 << 64) - 1


def philox4x64_10(ctr, key):
    """Philox4x64-10 block (Salmon, Moraes, Dror and Shaw, SC 2011), restated from its
    definition with Python integers: ten rounds of two 64 x 64 -> 128-bit products, the key
    advanced by the Weyl constants between rounds."""
    m0, m1 = 0xD2E7470EE14C6C93, 0xCA5A826395121157
    w0, w1 = 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B
    x = list(ctr)
    k0, k1 = key
    for _ in range(10):
        p0, p1 = m0 * x[0], m1 * x[2]
        x = [(p1 >> 64) ^ x[1] ^ k0, p1 & MASK, (p0 >> 64) ^ x[3] ^ k1, p0 & MASK]
        k0, k1 = (k0 + w0) & MASK, (k1 + w1) & MASK
    return x


def test_draws_follow_the_generator_definition():
    for seed, j in ((0, 0), (1805_06572, 1), (2**64 - 3, 0)):
        got = synth.philox_cn(seed, j, 9)
        for t in range(9):
            w = philox4x64_10([t, 0, 0, 0], [seed % 2**64, 1000 + j])
            u0 = ((w[0] >> 11) + 0.5) / 2.0**53
            u1 = ((w[1] >> 11) + 0.5) / 2.0**53
            r = np.sqrt(-np.log(u0))
            want = r * np.cos(2 * np.pi * u1) + 1j * (r * np.sin(2 * np.pi * u1))
            assert got[t] == want, (seed, j, t)


def test_draws_are_circular_complex_normal():
    b = synth.philox_cn(77, 1, 40000)
    assert abs(np.mean(np.abs(b) ** 2) - 1.0) < 0.03          # E|b|^2 = 1
    assert abs(np.mean(b)) < 0.02 and abs(np.mean(b * b)) < 0.03  # zero mean, circular
    assert abs(np.mean(b.real ** 2) - 0.5) < 0.02              # each part N(0, 1/2)
    # the two sources' streams differ
    assert not np.allclose(synth.philox_cn(77, 0, 8), synth.philox_cn(77, 1, 8))


def test_initial_values_follow_the_recipe():
    M, F, N, seed = 3, 6, 50, 4242
    y = synth.make_mixture(M, F, N, 0.1, 1.0, seed)["y"]
    v0, S0 = synth.init_params(y, seed, recipe="random")
    yd = y.astype(np.complex128)
    pw = (np.abs(yd) ** 2).sum(axis=2)
    for j in range(2):
        b = synth.philox_cn(seed, j, F * M).reshape(F, M)
        for f in range(F):
            S = np.outer(b[f], b[f].conj()) + np.eye(M)
            np.testing.assert_allclose(S0[j, f], S, rtol=1e-15, atol=1e-15)
            assert np.linalg.eigvalsh(S0[j, f]).min() > 1 - 1e-12      # b b^H + I >= I
            tr = np.real(np.trace(S))
            eps = 1e-12 * pw[f].mean()
            np.testing.assert_allclose(v0[j, f] * 2 * tr, np.maximum(pw[f], eps), rtol=1e-14)
