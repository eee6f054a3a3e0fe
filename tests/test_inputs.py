"""The seeded input generators: determinism, counter addressing and shapes."""
import math

import numpy as np

from paper_1905_02803_gb300 import inputs


def test_counter_based_streams_are_addressable():
    a = inputs.uniform(7, 3, 100)
    b = inputs.uniform(7, 3, 40, start=60)
    assert np.array_equal(a[60:], b)
    assert not np.array_equal(a, inputs.uniform(8, 3, 100))
    assert not np.array_equal(a, inputs.uniform(7, 4, 100))
    assert a.min() >= 0.0 and a.max() < 1.0


def test_splitmix64_reference_values():
    # splitmix64 from state 0: published first outputs of the generator
    z = np.array([0], dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = []
        s = z.copy()
        for _ in range(3):
            s = s + inputs._GAMMA
            out.append(int(inputs._mix(s)[0]))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_moments():
    x = inputs.normal(0, 5, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01


def test_turbulence_field_unit_rms_and_deterministic():
    f = inputs.turbulence_field((16, 12, 10), seed=3)
    g = inputs.turbulence_field((16, 12, 10), seed=3)
    assert np.array_equal(f, g)
    assert abs(math.sqrt((f ** 2).mean()) - 1.0) < 1e-12


def test_channel_field_uses_end_orders():
    f = inputs.channel_field(12, 10, 9, seed=0)
    assert f.shape == (9, 10, 12)
    assert np.isfinite(f).all()


def test_smooth7_sizes_and_batch():
    s = inputs.smooth7_sizes()
    assert len(s) == 64 and sum(n % 2 for n in s) == 16
    assert s[0] == 48 and s[-1] == 384
    dims = inputs.batch_dims(0)
    assert len(dims) == 64 and all(d in s for t in dims for d in t)


def test_device_generator_matches_the_numpy_one():
    """The torch form of the counter-based generator (used for full-size grids
    on the GPU) gives the numpy form's values bit for bit (here on the host)."""
    torch = __import__("pytest").importorskip("torch")
    a = inputs.uniform_field((5, 7, 9), 4, stream=2)
    b = inputs.uniform_field_device((5, 7, 9), 4, stream=2, device="cpu", dtype=np.float64, zchunk=2)
    assert isinstance(b, torch.Tensor) and np.array_equal(a, b.numpy())
    u = inputs.uniform(9, 3, 500, start=(1 << 33) + 7)
    v = inputs.uniform_torch(9, 3, (1 << 33) + 7, 500).numpy()
    assert np.array_equal(u, v)


def test_power_law_half_spectrum():
    S = inputs.power_law_half_spectrum((8, 6, 10), 3)
    assert S.shape == (8, 6, 6) and S[0, 0, 0] == 0
    assert np.all(np.abs(S.ravel()[1:]) > 0)  # dense
    # |S|^2 = |k|^(-5/3): (kx, ky, kz) = (3, -2, 1) sits at [1][4][3]
    k2 = 9 + 4 + 1
    assert math.isclose(abs(S[1, 4, 3]) ** 2, k2 ** (-5.0 / 6.0), rel_tol=1e-12)
    assert np.array_equal(S, inputs.power_law_half_spectrum((8, 6, 10), 3))


def test_plane_waves_rank_sum():
    w = inputs.plane_waves((6, 8, 10), 5, n_waves=16)
    wa, wk, wphi = inputs._wave_params((6, 8, 10), 5, 16)
    z, y, x = 2, 3, 7
    direct = sum(a * math.cos(2 * math.pi * (k[0] * x / 10 + k[1] * y / 8 + k[2] * z / 6) + p)
                 for a, k, p in zip(wa, wk, wphi))
    assert math.isclose(w[z, y, x], direct, rel_tol=1e-12, abs_tol=1e-12)
