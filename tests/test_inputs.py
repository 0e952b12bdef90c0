"""Seeded input generator: determinism, ranges and the coefficient recipes."""
import numpy as np

from paper_1410_5561_gb300 import inputs


def test_counter_based_and_deterministic():
    a = inputs.uniform01_range(0, 3, 0, 1000)
    b = inputs.uniform01_range(0, 3, 500, 500)
    assert np.array_equal(a[500:], b)  # value n depends only on (seed, stream, n)
    c = inputs.uniform01_range(1, 3, 0, 1000)
    d = inputs.uniform01_range(0, 4, 0, 1000)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.05


def test_mix_matches_splitmix64_definition():
    # The mixing function written out with Python integers (mod 2^64).
    M = (1 << 64) - 1

    def mix(z):
        z ^= z >> 30; z = (z * 0xBF58476D1CE4E5B9) & M
        z ^= z >> 27; z = (z * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    G = 0x9E3779B97F4A7C15
    seed, stream = 12345, 7
    key = mix((seed * G + stream) & M)
    want = [(mix((key + (n + 1) * G) & M) >> 11) * 2.0 ** -53 for n in range(16)]
    got = inputs.uniform01_range(seed, stream, 0, 16)
    assert np.array_equal(got, np.array(want))


def test_chunked_fill_equals_direct():
    out = np.empty((3, 5, 7), dtype=np.float32)
    inputs.fill_uniform(out, 9, 0, -1.0, 1.0)
    ref = (-1.0 + 2.0 * inputs.uniform01_range(9, 0, 0, out.size)).astype(np.float32)
    assert np.array_equal(out.ravel(), ref)


def test_coefficient_recipes_row_sums():
    c7 = inputs.coefs_7pt_var(0, 6, 5, 4)
    assert c7.shape == (7, 4, 5, 6) and (c7 > 0).all()
    assert np.allclose(c7.sum(axis=0), 0.95, rtol=0, atol=1e-14)
    c25 = inputs.coefs_25pt_var(0, 6, 5, 4)
    assert c25.shape == (13, 4, 5, 6) and (c25 > 0).all()
    assert np.allclose(c25[0] + 2 * c25[1:].sum(axis=0), 0.95, rtol=0, atol=1e-14)


def test_batch_shapes_inclusive_bounds():
    shp = inputs.batch_shapes(0, count=4000)
    arr = np.array(shp)
    assert arr[:, :3].min() == 32 and arr[:, :3].max() == 192
    assert arr[:, 3].min() == 10 and arr[:, 3].max() == 200
    assert inputs.batch_shapes(0) == inputs.batch_shapes(0)
    assert len(inputs.batch_shapes(0)) == 64


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, 1.0 + 3 * 2 ** -8, -0.95])
    r = inputs.round_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie -> even
    assert r[2] == 1.0 + 2 ** -7          # above the tie -> up
    assert r[3] == 1.0 + 4 * 2 ** -8      # tie -> even (up)
    assert abs(r[4] + 0.95) < 2 ** -8


def test_torch_generator_matches_numpy():
    torch = __import__("pytest").importorskip("torch")
    a = torch.empty(3, 7, 11, dtype=torch.float64)
    inputs.fill_uniform_torch(a, 5, 2, -1.0, 1.0, chunk=37)
    b = inputs.uniform(5, 2, (3, 7, 11), -1.0, 1.0)
    assert np.array_equal(a.numpy(), b)
    f = torch.empty(5, 5, 5, dtype=torch.float32)
    inputs.fill_uniform_torch(f, 0, 0, -1.0, 1.0)
    g = np.empty((5, 5, 5), dtype=np.float32)
    inputs.fill_uniform(g, 0, 0, -1.0, 1.0)
    assert np.array_equal(f.numpy(), g)


def test_box_and_device_recipes_equal_the_full_arrays():
    """Crops drawn on their own, and the torch versions of the recipes, give exactly the
    values of the full CPU arrays: full-size parity cases build the device grid with the
    torch recipe and hand the oracle a crop."""
    torch = __import__("pytest").importorskip("torch")
    nx, ny, nz, seed = 11, 9, 7, 4
    lo, hi = (2, 1, 3), (6, 9, 10)
    sl = np.s_[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
    assert np.array_equal(inputs.field_u0_box(seed, nx, ny, nz, lo, hi), inputs.field_u0(seed, nx, ny, nz)[sl])
    u = inputs.field_u0_torch(seed, nx, ny, nz, torch.float32, "cpu")
    assert np.array_equal(u.numpy(), inputs.field_u0(seed, nx, ny, nz).astype(np.float32))
    for kind, full in (("7pt_var", inputs.coefs_7pt_var), ("25pt_var", inputs.coefs_25pt_var)):
        c = full(seed, nx, ny, nz)
        assert np.array_equal(inputs.coefs_box(kind, seed, nx, ny, nz, lo, hi), c[(slice(None),) + sl])
        d = inputs.coefs_torch(kind, seed, nx, ny, nz, torch.float64, "cpu")
        assert np.array_equal(np.stack([x.numpy() for x in d]), c)
        b = inputs.coefs_torch(kind, seed, nx, ny, nz, torch.bfloat16, "cpu")
        bits = np.stack([x.view(torch.int16).numpy().view(np.uint16) for x in b])
        assert np.array_equal(bits, inputs.bf16_bits(c))
    full_x = (0, 2, 0), (4, 7, nx)
    c = inputs.coefs_25pt_var(seed, nx, ny, nz)
    got = inputs.coefs_box("25pt_var", seed, nx, ny, nz, *full_x)
    assert np.array_equal(got, c[:, 0:4, 2:7, :])
