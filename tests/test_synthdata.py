"""The shared input generator: published SplitMix64 outputs, counter access and ranges."""
import numpy as np

import synthdata as sd


def test_splitmix64_known_answers():
    # Published first outputs of the SplitMix64 reference generator seeded with 1234567.
    assert sd.splitmix64_sequence(1234567, 5) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_counter_draw_is_the_sequence():
    seed, stream = 99, 3
    seq = sd.splitmix64_sequence(sd.mix64_int(seed), 300)
    got = sd.draw(seed, stream, 0, np.arange(256, dtype=np.uint64))
    base = stream << 48
    # output number c of the sequence is mix64(s + (c+1)*GAMMA); with ctr = base + w
    for w in (0, 1, 7, 255):
        s = (sd.mix64_int(seed) + (base + w + 1) * sd.GAMMA) & sd.MASK64
        assert int(got[w]) == sd.mix64_int(s)
    # stream 0, point 0: counters 0..255 are the first 256 outputs of the plain sequence
    got0 = sd.draw(seed, 0, 0, np.arange(256, dtype=np.uint64))
    assert [int(v) for v in got0] == seq[:256]


def test_points_random_access_and_ranges():
    mix = sd.make_mixture(7, 16)
    a = sd.points(mix, sd.STREAM_BASE, 0, 5000)
    b = sd.points(mix, sd.STREAM_BASE, 1234, 10)
    assert a.dtype == np.uint8 and a.shape == (5000, 128)
    assert np.array_equal(a[1234:1244], b)
    assert not np.array_equal(a[:10], sd.points(mix, sd.STREAM_QUERY, 0, 10))
    assert mix.cum[-1] == 1 << 32 and np.all(np.diff(mix.cum.astype(np.int64)) > 0)
    assert mix.B.min() >= -3 and mix.B.max() <= 3
    assert 3 <= mix.sigma.min() and mix.sigma.max() <= 6


def test_points_scalar_definition():
    """Recompute one point with Python ints straight from the module docstring."""
    mix = sd.make_mixture(5, 8)
    n, stream = 321, sd.STREAM_LEARN
    seedk = sd.mix64_int(mix.seed)

    def word(w):
        ctr = (stream << 48) | (n << 8) | w
        return sd.mix64_int(seedk + (ctr + 1) * sd.GAMMA)

    r = word(0) >> 32
    comp = next(c for c in range(mix.n_comp) if int(mix.cum[c]) > r)
    z = []
    for w in range(1, 1 + sd.N_FACTORS // 2 + mix.dim // 2):
        v = word(w)
        for half in (v & 0xFFFFFFFF, v >> 32):
            z.append(sum((half >> (8 * i)) & 0xFF for i in range(4)) - 510)
    lat, noise = z[:sd.N_FACTORS], z[sd.N_FACTORS:]
    x = []
    for d in range(mix.dim):
        a = int(mix.sigma[comp]) * sum(int(mix.B[d][f]) * lat[f] for f in range(sd.N_FACTORS)) + sd.NOISE * noise[d]
        x.append(min(255, max(0, int(mix.mu[comp][d]) + (a + 83) // 166)))
    assert list(sd.points(mix, stream, n, 1)[0]) == x
