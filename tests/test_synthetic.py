"""The seeded input generators: SplitMix64 against its published test vector, determinism."""
import numpy as np

import synthetic as S


def test_splitmix64_reference_vector():
    # SplitMix64 started from state 0: the first outputs of the published generator
    z = S.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_statistics():
    u = S.uniform(123, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    n = S.normal(321, 200000)
    assert abs(n.mean()) < 1e-2 and abs(n.std() - 1.0) < 1e-2


def test_generators_are_deterministic():
    assert np.array_equal(S.uniform(5, (3, 4)), S.uniform(5, (3, 4)))
    a = S.cfg3_ragged()
    b = S.cfg3_ragged()
    assert a == b and len(a) == 200
    assert {d["n"] for d in a} <= set(S.CFG3_SIZES)


def test_smooth_phase_screen_std():
    s = S.smooth_noise(9, (64, 64), 4.0, 1.0)
    assert abs(s.std() - 1.0) < 1e-12
