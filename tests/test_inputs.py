"""The seeded input generators: the recipes they promise (no method arithmetic)."""
import numpy as np

from paper_2403_18466_gb300 import inputs


def test_random_field_is_divergence_free_with_requested_rms():
    rho, ux, uy = inputs.random_velocity_field(64, 48, seed=1, k0=8.0, urms=0.02)
    assert np.allclose(rho, 1.0)
    assert np.isclose(np.sqrt(0.5 * np.mean(ux ** 2 + uy ** 2)), 0.02, rtol=1e-12)
    assert abs(ux.mean()) < 1e-15 and abs(uy.mean()) < 1e-15
    kx = 2j * np.pi * np.fft.fftfreq(48)[None, :]
    ky = 2j * np.pi * np.fft.fftfreq(64)[:, None]
    div = np.fft.ifft2(kx * np.fft.fft2(ux) + ky * np.fft.fft2(uy)).real
    assert np.abs(div).max() < 1e-14
    # seeded: same seed, same field; other seed, other field
    assert np.array_equal(ux, inputs.random_velocity_field(64, 48, seed=1)[1])
    assert not np.array_equal(ux, inputs.random_velocity_field(64, 48, seed=2)[1])


def test_xavier_bounds_and_packing():
    th = inputs.xavier_mlp(3)
    assert th.size == inputs.mlp_nparams() == 5385
    W1, b1, W2, b2, W3, b3 = inputs.unpack_mlp(th)
    assert np.abs(W1).max() <= np.sqrt(6 / 73) and np.abs(W2).max() <= np.sqrt(6 / 128)
    assert not b1.any() and not b2.any() and not b3.any()
