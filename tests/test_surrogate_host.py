"""Host-side pieces of the surrogate search (no GPU): the mirrored encoding
formed on encoded grids equals encoding the mirrored robots, row for row."""
import numpy as np

from paper_1911_10274_gb300 import surrogate as S


def test_mirrored_encoding_equals_encoding_the_mirrored_robots():
    rng = np.random.default_rng(4)
    ms = [S.random_morph(rng) for _ in range(7)]
    f = rng.normal(0, 0.03, 7)
    am, af = S.mirrored(ms, f)
    Xa = S.encode(am)
    Xb, fb = S.mirrored_encoded(S.encode(ms), f)
    assert Xa.dtype == Xb.dtype and np.array_equal(Xa, Xb)
    assert np.array_equal(af, fb)


def test_mirror_negates_the_x_displacement_only():
    rng = np.random.default_rng(5)
    ms = [S.random_morph(rng) for _ in range(3)]
    _, y = S.mirrored_encoded(S.encode(ms), np.array([0.1, -0.2, 0.3]))
    assert np.array_equal(y.reshape(3, 4), np.array([[0.1, 0.1, -0.1, -0.1], [-0.2, -0.2, 0.2, 0.2],
                                                     [0.3, 0.3, -0.3, -0.3]]))
