"""The seeded input recipes are deterministic and have the stated shapes."""
import numpy as np

import workloads as W


def test_random_state_unit_columns_and_seeded():
    a = W.random_state(1000, 5, seed=3)
    b = W.random_state(1000, 5, seed=3)
    assert a.shape == (1000, 5) and np.array_equal(a, b)
    assert np.allclose(np.linalg.norm(a, axis=0), 1.0, atol=1e-14)
    assert W.random_state(64, 1, seed=1).shape == (64,)


def test_wavepacket_is_a_unit_gaussian_at_two():
    D = 4096
    psi = W.wavepacket(D)
    L = W.dvr_default_L(D)
    x = -L + (2 * L / (D - 1)) * np.arange(D)
    p = np.abs(psi) ** 2
    assert abs(p.sum() - 1) < 1e-14
    assert abs((p * x).sum() - 2.0) < 1e-12              # <x> = 2
    assert abs((p * (x - 2) ** 2).sum() - 0.5) < 1e-9    # variance 1/2 of exp(-(x-2)^2/2)^2


def test_batch_recipe():
    probs = W.batch_problems(256)
    assert probs == W.batch_problems(256)
    D = np.array([p[0] for p in probs])
    nv = np.array([p[1] for p in probs])
    assert len(probs) == 256 and [p[2] for p in probs] == list(range(256))
    assert D.min() >= 1024 and D.max() <= 32768 and np.all(D % 128 == 0)
    assert nv.min() >= 1 and nv.max() <= 16
    # log-uniform: about half of the draws below the geometric midpoint
    assert 0.35 < np.mean(D < np.sqrt(1024 * 32768)) < 0.65
