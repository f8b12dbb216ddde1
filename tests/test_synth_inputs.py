"""Host checks of the seeded input generators the workloads and the oracle share (they hold no
arithmetic of the method): determinism, and the distributions the recipes state."""
import numpy as np

import synth


def test_stretch_ball_is_symmetric_inside_the_ball_and_uniform_in_volume():
    U = synth.stretch_ball(1004, 20000, 0.3)
    assert np.array_equal(U, synth.stretch_ball(1004, 20000, 0.3))  # counter-based: reproducible
    assert np.allclose(U, np.swapaxes(U, 1, 2))
    r = np.linalg.norm((U - np.eye(3)).reshape(-1, 9), axis=1)
    assert r.max() <= 0.3 + 1e-12
    # uniform in the 6-dimensional ball: P(r <= s) = (s / 0.3)^6
    for s in (0.15, 0.25, 0.28):
        assert abs((r <= s).mean() - (s / 0.3) ** 6) < 0.01
    # isotropic in Mandel form: each of the 6 components has the same variance
    v = np.stack([U[:, 0, 0] - 1, U[:, 1, 1] - 1, U[:, 2, 2] - 1,
                  np.sqrt(2) * U[:, 1, 2], np.sqrt(2) * U[:, 0, 2], np.sqrt(2) * U[:, 0, 1]], 1)
    var = v.var(axis=0)
    assert np.abs(var / var.mean() - 1).max() < 0.05
    assert np.abs(v.mean(axis=0)).max() < 0.005
    # a later slice of the same stream continues it (keys are absolute indices)
    assert np.array_equal(synth.stretch_ball(1004, 10, 0.3, first=5), U[5:15])


def test_fixed_rve12_is_two_phase_with_the_recorded_fraction():
    phase, phi = synth.fixed_rve12()
    assert phase.shape == (12 ** 3,) or phase.size == 12 ** 3
    frac = float((np.asarray(phase) == 1).mean())
    assert set(np.unique(phase)) <= {0, 1}
    assert 0.1 <= phi <= 0.3 and 0.0 < frac < 0.5
