"""Pins for the oracle kick-drift and the full compressed step: a free
particle moves exactly c_drift v, momentum is conserved across a step, and a
step from compressed state round-trips through the codec of Sec. 2.4."""
import numpy as np

from oracle import codec, step

G = 1.0 / (4 * np.pi)


def _cfg(**kw):
    c = dict(n_fine=32, coarse_ratio=1, tile=32, buffer=0, cmp_ratio=4, vel_bits=16, G=G,
             mass=(8.0, 0.04), r_split=0.0, r_cut=0.0)
    c.update(kw)
    return c


def test_free_particle_drift_and_wrap():
    x = np.array([[1.0, 2.0, 31.5]])
    v = np.array([[0.5, -3.0, 1.0]])
    x1, v1 = step.kick_drift(x, v, np.zeros((1, 3)), 1.0, 2.0, 32)
    np.testing.assert_array_equal(v1, v)
    np.testing.assert_array_equal(x1, [[2.0, 28.0, 1.5]])


def test_zero_gravity_step_is_pure_drift():
    rng = np.random.default_rng(21)
    cfg = _cfg(G=0.0)
    xs = [(rng.random((100, 3)) * 32).astype(np.float32), (rng.random((400, 3)) * 32).astype(np.float32)]
    vs = [rng.standard_normal((100, 3)).astype(np.float32), rng.standard_normal((400, 3)).astype(np.float32)]
    codes = [codec.compress(x, v, 32, 8, 16) for x, v in zip(xs, vs)]
    new, states = step.step(codes, cfg, 1.0, 1.0)
    for c, (x1, v1), c_new in zip(codes, states, new):
        xd, vd = codec.decompress(c, 32)
        np.testing.assert_array_equal(v1, vd)
        np.testing.assert_allclose(x1, np.mod(xd.astype(np.float64) + vd, 32), atol=0)
        assert c_new.n == c.n and c_new.vmax == np.max(np.abs(vd))


def test_step_conserves_momentum():
    rng = np.random.default_rng(22)
    cfg = _cfg()
    xs = [(rng.random((150, 3)) * 32).astype(np.float32), (rng.random((600, 3)) * 32).astype(np.float32)]
    vs = [rng.standard_normal((150, 3)).astype(np.float32), rng.standard_normal((600, 3)).astype(np.float32)]
    codes = [codec.compress(x, v, 32, 8, 16) for x, v in zip(xs, vs)]
    _, states = step.step(codes, cfg, 0.5, 1.0)
    p0 = sum(m * codec.decompress(c, 32)[1].astype(np.float64).sum(0) for m, c in zip(cfg["mass"], codes))
    p1 = sum(m * s[1].sum(0) for m, s in zip(cfg["mass"], states))
    np.testing.assert_allclose(p1, p0, atol=1e-11)


def test_step_output_decodes_within_codec_bounds():
    rng = np.random.default_rng(23)
    cfg = _cfg(coarse_ratio=4, tile=8, buffer=8, r_split=0.8, r_cut=4.0)
    xs = [(rng.random((120, 3)) * 32).astype(np.float32), (rng.random((480, 3)) * 32).astype(np.float32)]
    vs = [rng.standard_normal((120, 3)).astype(np.float32), rng.standard_normal((480, 3)).astype(np.float32)]
    codes = [codec.compress(x, v, 32, 8, 16) for x, v in zip(xs, vs)]
    new, states = step.step(codes, cfg, 1.0, 1.0)
    for c_new, (x1, v1) in zip(new, states):
        xd, vd = codec.decompress(c_new, 32)
        cell = np.floor(step.to_f32_positions(x1, 32) / 4).astype(np.int64)
        perm = np.argsort(cell[:, 0] + 8 * (cell[:, 1] + 8 * cell[:, 2]), kind="stable")
        assert np.max(np.abs(xd - x1[perm])) <= 4 / 512 + 1e-5
        assert np.max(np.abs(vd - v1[perm])) <= c_new.vmax / 2 ** 16 * 1.001 + 1e-6
