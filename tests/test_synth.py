"""The shared seeded input generator: splitmix64 against its published reference outputs."""
import numpy as np

from paper_1403_4661_gb300 import synth


def test_splitmix64_reference_values():
    # reference outputs of splitmix64 (Steele, Lea, Flood 2014; Vigna's C reference code)
    assert [int(x) for x in synth.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert int(synth.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    # counter form: any window of the stream equals the same slice of a longer draw
    np.testing.assert_array_equal(synth.splitmix64(9, 4, start=10), synth.splitmix64(9, 20)[10:14])


def test_distributions_and_shapes():
    u = synth.uniform_pm1(3, 200000)
    assert -1.0 <= u.min() and u.max() < 1.0 and abs(u.mean()) < 0.01
    g = synth.normal(4, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    c = synth.decaying_coeffs(8, 3, 1)
    assert c.shape == (3, 64) and c.dtype == np.complex128
    L = synth.loguniform_bandlimits(512, 32, 1024, 5)
    assert L.min() >= 32 and L.max() <= 1024
    np.testing.assert_array_equal(synth.uniform_coeffs(5, 2, 7), synth.uniform_coeffs(5, 2, 7))
