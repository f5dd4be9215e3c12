"""The seeded input generator: SplitMix64 stream, Gaussian moments, SU(3) links."""
import numpy as np

import synth

M64 = 2**64 - 1


def _splitmix64_sequential(seed, n):
    """Sequential SplitMix64 (Steele, Lea, Flood 2014): state += gamma; mix(state)."""
    out, s = [], seed
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_counter_matches_sequential():
    for seed in (0, 1, 1001, 2**63 + 5):
        seq = _splitmix64_sequential(seed, 40)
        assert [synth.splitmix64_at(seed, n) for n in range(40)] == seq
    assert synth.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF   # published first output for seed 0


def test_gaussian_moments_and_determinism():
    g = synth.gaussian(1_000_001, seed=2001)
    assert abs(g.mean()) < 5e-3 and abs(g.std() - 1) < 5e-3
    assert np.array_equal(g[:1000], synth.gaussian(1000, seed=2001))


def test_su3_links_unitary_det_one_and_smooth():
    u = synth.su3(20000, 0.2, seed=1001)
    eye = np.eye(3)
    uu = u @ u.conj().transpose(0, 2, 1)
    assert np.max(np.abs(uu - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(u) - 1)) < 1e-14
    # exp(i eps H) with eps = 0.2 stays near the identity; a larger eps moves further away
    d02 = np.mean(np.abs(u - eye))
    d15 = np.mean(np.abs(synth.su3(20000, 1.5, seed=1001) - eye))
    assert 0.02 < d02 < 0.3 and d15 > 2 * d02


def test_gauge_layout_and_seed_independence():
    dims = (4, 2, 2, 4)
    u = synth.gauge(dims, seed=1064)
    assert u.shape == (64, 4, 3, 3)
    flat = synth.su3(4 * 64, 0.2, seed=1064)
    assert np.array_equal(u.reshape(-1, 3, 3), flat)
    assert not np.array_equal(u, synth.gauge(dims, seed=1065))
