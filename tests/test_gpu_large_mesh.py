"""Two-level meshes whose coarse edge exceeds one shared-memory plane (192^3,
256^3, 384^3 coarse; 768^3 to 1536^3 fine): the row / column FFT passes of
the periodic long-range solve against the oracle -- the whole 192^3 mesh in
float and fixed point, sampled Fourier modes at 256^3 and 384^3 -- and the
fused step on a 768^3 mesh against the plain path bit for bit in fixed point."""
import gc

import numpy as np
import pytest
import torch

from oracle import solve
from synth import make_workload
from tests.helpers import oracle_codes_from_lib, records, rel_rms

pytestmark = pytest.mark.gpu

G = 1.0 / (4 * np.pi)


def _cfg(nf, counts=(1000, 8000), **kw):
    c = dict(n_fine=nf, coarse_ratio=4, tile=64, buffer=16, cmp_ratio=4, vel_bits=16, G=G, mass=(8.0, 0.04),
             count=counts, r_split=14.0 / 4.5, r_cut=14.0)
    c.update(kw)
    return c


def _need(gbytes):
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < gbytes * 1e9:
        pytest.skip(f"needs {gbytes} GB of free device memory, {free / 1e9:.0f} GB free")


def _coarse_solve(pm, rc):
    """Solve with the given coarse density and an empty fine mesh; returns acc_coarse."""
    rf = torch.zeros((pm.n_fine,) * 3, dtype=rc.dtype, device="cuda")
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    pm.check()
    del rf, af
    return ac


def test_coarse_192_solve_matches_oracle():
    from paper_1611_01545_gb300 import PM
    _need(40)
    g = torch.Generator(device="cuda").manual_seed(192)
    for mode in (0, 1):
        pm = PM(_cfg(768, deposit_mode=mode))
        assert pm.n_coarse == 192
        if mode == 0:
            rc = torch.randn((192,) * 3, device="cuda", generator=g)
            M = rc.cpu().numpy().astype(np.float64)
        else:
            # fixed point: masses in units of 2^-32
            rc = torch.randint(-(1 << 34), 1 << 34, (192,) * 3, device="cuda", generator=g, dtype=torch.int64)
            M = rc.cpu().numpy().astype(np.float64) * 2.0 ** -32
        ac = _coarse_solve(pm, rc)
        ref = solve.accel_periodic(M, 4.0, G, 14.0 / 4.5)
        assert rel_rms(ac.cpu().numpy(), ref) < 1e-5
        pm.close()


@pytest.mark.parametrize("nf", [1024, 1536])
def test_large_coarse_solve_sampled_modes(nf):
    from paper_1611_01545_gb300 import PM
    nc = nf // 4
    _need(40 if nf == 1024 else 125)
    pm = PM(_cfg(nf, tile_batch=64))
    assert pm.n_coarse == nc
    g = torch.Generator(device="cuda").manual_seed(nc)
    rc = torch.rand((nc,) * 3, device="cuda", generator=g)
    ac = _coarse_solve(pm, rc).cpu().numpy()
    pm.close()
    M = rc.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(nc)
    # long waves (|m| <= 12, negative mode numbers included), where the long-range
    # force lives: far above the float32 round-off that the transforms spread
    # over all modes
    modes = [(1, 0, 0), (0, 1, 2), (3, 2, 1), (nc - 2, 1, 5), (7, nc - 4, 11), (0, nc - 1, nc - 3)]
    modes += [tuple(int(v) for v in rng.integers(0, 12, 3)) for _ in range(4)]
    for m in modes:
        ref = solve.accel_mode(M, 4.0, G, 14.0 / 4.5, m)
        got = np.array([solve.dft_mode(ac[d], m) for d in range(3)])
        scale = np.abs(ref).max()
        if scale == 0.0:
            continue
        assert np.all(np.abs(got - ref) <= 1e-4 * scale), (m, got, ref)


def test_fused_step_equals_plain_path_768():
    from paper_1611_01545_gb300 import PM
    _need(40)
    w = make_workload("two_level768")
    for mode in (1, 0):
        pm = PM(dict(w.config(), deposit_mode=mode))
        codes = []
        for s in range(2):
            x = torch.from_numpy(w.x[s]).cuda()
            v = torch.from_numpy(w.v[s]).cuda()
            codes.append(pm.compress(s, x, v, out=pm.empty_codes(x.shape[0], esc_cap=x.shape[0] // 255 + 1)))
        out = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in codes]
        pm.step(codes, out, 1.0, 1.0)
        pm.check()
        nc = w.n_fine // 4
        if mode == 0:
            # float: particles conserved per species, status clean
            for s in range(2):
                a = oracle_codes_from_lib(out[s], nc, w.vel_bits)
                assert a.counts().sum() == w.counts[s]
            pm.close()
            continue
        xs, vs = zip(*[pm.decompress(s, codes[s]) for s in range(2)])
        rc, rf = pm.density(list(xs), fixed=True)
        ac, af = pm.zeros_acc()
        pm.solve(rc, rf, ac, af)
        for s in range(2):
            x, v = xs[s].clone(), vs[s].clone()
            pm.kick_drift(x, v, ac, af, 1.0, 1.0)
            plain = pm.compress(s, x, v, out=pm.empty_codes(x.shape[0], esc_cap=out[s].esc.shape[0]))
            pm.check()
            a = oracle_codes_from_lib(out[s], nc, w.vel_bits)
            b = oracle_codes_from_lib(plain, nc, w.vel_bits)
            assert a.vmax == b.vmax and a.counts().sum() == w.counts[s]
            np.testing.assert_array_equal(a.cnt, b.cnt)
            np.testing.assert_array_equal(records(a), records(b))
        del xs, vs, rc, rf, ac, af
        pm.close()
