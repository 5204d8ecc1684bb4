"""Pins for the bound mode of the recompressed velocity scale (vmax_mode 1)
and for the assembled fine force mesh it is taken over: the assembled mesh
interpolated globally reproduces every particle's home-tile interpolation;
the bound holds for every kicked velocity and is attained, up to half a
velocity bin, by a particle sitting on the extreme node of both meshes."""
import numpy as np
import pytest

from oracle import codec, mesh, step
from synth import make_workload


def _two_level_small():
    w = make_workload("two_level64", n_cdm=8, n_nu=12)
    return w, w.config()


def test_assembled_fine_mesh_equals_home_tile_interpolation():
    w, cfg = _two_level_small()
    xs = [np.asarray(x, np.float64) for x in w.x]
    af = step.fine_accel_mesh(xs, cfg)
    home = step.fine_accel(xs, cfg)
    for x, a in zip(xs, home):
        np.testing.assert_allclose(mesh.cic_interp(af, x, w.n_fine), a, rtol=0, atol=1e-12 * np.max(np.abs(a)))


@pytest.mark.parametrize("name", ["single64", "two_level64"])
def test_bound_holds_for_every_kicked_velocity(name):
    w = make_workload(name, n_cdm=8, n_nu=12)
    cfg = w.config()
    n_cmp = w.n_fine // 4
    codes = [codec.compress(w.x[s], w.v[s], w.n_fine, n_cmp, w.vel_bits) for s in range(2)]
    for ck in (1.0, -3.0):
        new, states = step.step(codes, cfg, ck, 0.5, vmax_mode=1)
        exact, _ = step.step(codes, cfg, ck, 0.5, vmax_mode=0)
        for s in range(2):
            v1 = states[s][1]
            assert np.max(np.abs(v1)) <= float(new[s].vmax)
            assert float(new[s].vmax) >= float(exact[s].vmax)   # exact max never above the bound


def test_bound_is_attained_on_the_extreme_nodes():
    # coarse mesh (ratio 4) with its largest |a| at coarse node C, fine mesh with
    # its largest |a| at fine node 4C; a particle at fine position 4C whose
    # decoded velocity is the largest positive code sees both maxima.
    rng = np.random.default_rng(3)
    n, rc = 16, 4
    nc = n // rc
    ac = rng.uniform(-1, 1, (3, nc, nc, nc))
    af = rng.uniform(-1, 1, (3, n, n, n))
    C = np.array([1, 2, 3])           # x, y, z
    ac[1, C[2], C[1], C[0]] = 2.5
    af[1, rc * C[2], rc * C[1], rc * C[0]] = 1.75
    vmax_in, ck, bits = np.float32(0.8), 1.5, 16
    half = 2 ** (bits - 1)
    q = np.array([[half, 2 * half - 1, half]])
    v = codec.velocity_decode(q, vmax_in, bits).astype(np.float64)
    x = (rc * C).astype(np.float64)[None, :]
    a = mesh.cic_interp(ac, x / rc, nc) + mesh.cic_interp(af, x, n)
    v1 = v + ck * a
    bound = float(step.vmax_bound(vmax_in, [ac, af], ck))
    assert abs(v1[0, 1]) <= bound
    assert bound - abs(v1[0, 1]) <= 0.5 * float(vmax_in) / half + 1e-6
