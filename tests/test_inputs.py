"""The seeded synthetic inputs: same seed, same array; shapes and value ranges of the workload recipes."""
import numpy as np

import synth


def test_inputs_are_deterministic():
    a = synth.gaussian_beam_with_rectangles(6, seed=5)
    b = synth.gaussian_beam_with_rectangles(6, seed=5)
    assert a.dtype == np.complex64 and a.shape == (64, 64) and np.array_equal(a, b)
    assert not np.array_equal(a, synth.gaussian_beam_with_rectangles(6, seed=6))
    fx1, gy1 = synth.separable_phase_factors(8)
    fx2, gy2 = synth.separable_phase_factors(8)
    assert fx1.shape == (8, 256) and np.array_equal(fx1, fx2) and np.array_equal(gy1, gy2)
    assert synth.batched_item_specs(count=16) == synth.batched_item_specs(count=16)


def test_recipe_ranges():
    # beam times binary aperture: magnitudes in [0, 1], some pixels blocked
    a = np.abs(synth.gaussian_beam_with_rectangles(7, seed=11))
    assert a.max() <= 1.0 + 1e-6 and (a == 0).any()
    # batched items: n in 8..12 and chi in {16, 32, 64}
    specs = synth.batched_item_specs(count=64)
    assert all(8 <= s["n"] <= 12 and s["chi"] in (16, 32, 64) for s in specs)
    # phase-mask factors have unit modulus
    mx, my = synth.smooth_random_phase_mask_factors(8, seed=3, strength=0.5)
    assert np.allclose(np.abs(mx), 1.0) and np.allclose(np.abs(my), 1.0)
