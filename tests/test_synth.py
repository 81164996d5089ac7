"""The seeded input generators: the device vortex-sum generator of the
uneven batch agrees with the NumPy one (same parameter draws, untruncated
Gaussians), and the batch follows its stated recipe."""
import numpy as np

from paper_2510_25143_gb300 import synth


def test_device_vortex_sum_matches_numpy_without_noise():
    a = synth.vortex_sum_device(37, 52, 4, seed=5, n_vortex=4, drift=0.6, noise=0.0, device="cpu").numpy()
    b = synth.vortex_sum(37, 52, 4, seed=5, n_vortex=4, drift=0.6, noise=0.0)
    # the NumPy generator truncates each vortex at 6 radii: exp(-18) relative
    assert np.abs(a - b).max() <= 1e-6 * max(1.0, np.abs(b).max())


def test_device_vortex_sum_is_seeded():
    a = synth.vortex_sum_device(20, 24, 3, seed=7, n_vortex=3, drift=0.5, device="cpu").numpy()
    b = synth.vortex_sum_device(20, 24, 3, seed=7, n_vortex=3, drift=0.5, device="cpu").numpy()
    c = synth.vortex_sum_device(20, 24, 3, seed=8, n_vortex=3, drift=0.5, device="cpu").numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    noise = a - synth.vortex_sum_device(20, 24, 3, seed=7, n_vortex=3, drift=0.5, noise=0.0, device="cpu").numpy()
    assert 0.5e-3 < noise.std() < 2e-3


def test_batch_specs_follow_the_recipe():
    specs = synth.batch_specs(64, seed=2000)
    assert len(specs) == 64 and specs == synth.batch_specs(64, seed=2000)
    for d in specs:
        assert 128 <= d["H"] <= 1024 and 128 <= d["W"] <= 1024
        assert d["H"] % 16 == 0 and d["W"] % 16 == 0
        assert 10 <= d["T"] <= 200
        assert 0.2 <= d["drift"] <= 1.5 and d["n_vortex"] == max(6, d["H"] * d["W"] // 2048)
    assert len({d["seed"] for d in specs}) == 64
    assert len({(d["H"], d["W"], d["T"]) for d in specs}) > 32  # uneven
