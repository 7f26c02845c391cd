"""The seeded input generator shared by the oracle, the GPU tests and the bench: SplitMix64
(Steele, Lea and Flood 2014) against the reference implementation's published outputs, the
double mapping, and the two distributions' supports."""
import numpy as np

from paper_2003_01836_gb300 import inputs


def test_splitmix64_reference_outputs():
    # first five outputs of the reference splitmix64 generator seeded with 1234567
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in inputs.splitmix64(1234567, 0, 5)] == want
    # counter-based: any window of the stream is the same draws
    assert [int(v) for v in inputs.splitmix64(1234567, 2, 3)] == want[2:]


def test_uniform01_mapping():
    u = inputs.uniform01(1234567, 0, 5)
    raw = inputs.splitmix64(1234567, 0, 5)
    assert np.array_equal(u, (raw >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    assert np.all((u >= 0.0) & (u < 1.0))


def test_distributions():
    x, y, z, q = inputs.uniform_cube(50000, inputs.SEED_BASE)
    for a in (x, y, z, q):
        assert np.all((a >= -1.0) & (a < 1.0))
        assert abs(a.mean()) < 0.02
    x, y, z, q = inputs.plummer(50000, inputs.SEED_BASE + 2)
    r = np.sqrt(x * x + y * y + z * z)
    assert np.all(r <= 10.0 * (1 + 1e-12)) and np.all((q >= -1.0) & (q < 1.0))
    # enclosed fraction at r = 1 of the truncated Plummer sphere: M(1) / M(10)
    frac = (1.0 / 2.0 ** 1.5) / inputs.PLUMMER_MASS_AT_RMAX
    assert abs(np.mean(r <= 1.0) - frac) < 0.01
    # the chunked generation equals a single stream: particle i takes draws 4i .. 4i+3
    u = inputs.uniform01(inputs.SEED_BASE, 4 * 777, 4)
    xc, yc, zc, qc = inputs.uniform_cube(1000, inputs.SEED_BASE)
    assert np.array_equal(np.array([xc[777], yc[777], zc[777], qc[777]]), 2.0 * u - 1.0)
