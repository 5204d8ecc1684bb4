"""The largest one-GPU workload at full size: 1536^3 fine mesh (384^3 coarse,
13,824 tiles of 96^3), 768^3 CDM + 1536^3 neutrinos = 4.08e9 particles with
16-bit velocities, built on the device (bench.build_largest_codes), in the
launch configuration bench.py times for it.  Checked against what the oracle
can compute piece by piece and properties that hold at any size: particle and
mass conservation of the fused deposit, the fused density of a sub-box
against the oracle's CIC deposit of the decoded particles around it, the
384^3 long-range solve at sampled Fourier modes, one tile solve, sampled
force interpolations, and the fused step's status, counts and v_max."""
import gc

import numpy as np
import pytest
import torch

from oracle import codec, mesh, solve
from tests.helpers import rel_rms

pytestmark = pytest.mark.gpu

NEED_GB = 262


def _decode_cells(c, cells_xyz, cnt_host, off_host, n_fine, n_cmp, vel_bits):
    """Decoded float32 positions and velocities of every particle in the given
    compression cells (oracle decode of the codes copied from the device)."""
    idx, cxyz = [], []
    for (cx, cy, cz) in cells_xyz:
        cell = cx + n_cmp * (cy + n_cmp * cz)
        k = int(cnt_host[cell])
        idx.append(np.arange(off_host[cell], off_host[cell] + k))
        cxyz.append(np.repeat(np.array([[cx, cy, cz]]), k, axis=0))
    idx = np.concatenate(idx)
    cxyz = np.concatenate(cxyz)
    ti = torch.from_numpy(idx).cuda()
    q = c.pos[ti, :3].cpu().numpy().astype(np.int64)
    qv = c.vel[ti, :3].cpu().numpy()
    qv = qv.view(np.uint16).astype(np.int64) if vel_bits == 16 else qv.astype(np.int64)
    x = codec.position_decode(cxyz, q, n_fine, n_cmp)
    v = codec.velocity_decode(qv, np.float32(c.vmax.item()), vel_bits)
    return x, v


def test_largest_workload_full_size():
    import bench
    from paper_1611_01545_gb300 import PM
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_GB * 1e9:
        pytest.skip(f"needs {NEED_GB} GB of free device memory, {free / 1e9:.0f} GB free")
    cfg = bench.largest_config()
    nf, ncmp = cfg["n_fine"], cfg["n_fine"] // 4
    pm = PM(cfg)
    codes = bench.build_largest_codes(pm, torch)
    counts = cfg["count"]
    cnts, offs = [], []
    for s in range(2):
        assert codes[s].n == counts[s]
        cnt = codes[s].cnt.cpu().numpy().astype(np.int64)
        ne = int(codes[s].n_esc.item())
        esc = codes[s].esc[:ne].cpu().numpy().view(np.uint32)
        cnt[esc[:, 0].astype(np.int64)] = esc[:, 1]
        assert cnt.sum() == counts[s]
        cnts.append(cnt)
        offs.append(np.concatenate([[0], np.cumsum(cnt)]))

    # fused deposit: mass conservation on both meshes, and a sub-box against the oracle
    rc, rf = pm.zeros_meshes()
    pm.deposit_codes(codes, rc, rf)
    pm.check()
    total = sum(counts[s] * cfg["mass"][s] for s in range(2))
    assert abs(torch.sum(rf, dtype=torch.float64).item() - total) <= 1e-5 * total
    assert abs(torch.sum(rc, dtype=torch.float64).item() - total) <= 1e-5 * total
    c0 = np.array([101, 57, 230])            # compression cells of the sub-box: c0 .. c0 + 3
    k = 3
    cells = [(int(c0[0] + i), int(c0[1] + j), int(c0[2] + l))
             for l in range(-1, k + 1) for j in range(-1, k + 1) for i in range(-1, k + 1)]
    lo = (c0 - 1) * 4                        # fine origin of the local mesh
    m = (k + 2) * 4 + 1
    sub = np.zeros((m, m, m))
    xs_sample = []
    for s in range(2):
        x, _ = _decode_cells(codes[s], cells, cnts[s], offs[s], nf, ncmp, 16)
        sub += mesh.cic_deposit(x.astype(np.float64) - lo, cfg["mass"][s], m)
        xs_sample.append(x)
    a, b = c0 * 4, (c0 + k) * 4              # interior fine nodes: all their particles were decoded
    got = rf[a[2]:b[2], a[1]:b[1], a[0]:b[0]].cpu().numpy()
    assert rel_rms(got, sub[4:4 + 4 * k, 4:4 + 4 * k, 4:4 + 4 * k]) < 1e-5

    # solve: the 384^3 long-range mesh at sampled long-wave modes, one tile, interpolation
    ac, af = pm.zeros_acc()
    pm.solve(rc, rf, ac, af)
    pm.check()
    M = rc.cpu().numpy().astype(np.float64)
    acc_c = ac.cpu().numpy()
    for mm in [(1, 0, 0), (0, 2, 1), (3, 1, 2), (ncmp - 2, 4, 1), (5, ncmp - 3, 7)]:
        ref = solve.accel_mode(M, 4.0, cfg["G"], cfg["r_split"], mm)
        gotm = np.array([solve.dft_mode(acc_c[d], mm) for d in range(3)])
        assert np.all(np.abs(gotm - ref) <= 1e-4 * np.abs(ref).max()), (mm, gotm, ref)
    del M
    t, bb = cfg["tile"], cfg["buffer"]
    T = t + 2 * bb
    tix = np.array([5, 7, 11])
    org = tix * t - bb
    rng_idx = [torch.from_numpy((org[d] + np.arange(T)) % nf).cuda() for d in range(3)]
    win = rf[rng_idx[2]][:, rng_idx[1]][:, :, rng_idx[0]].cpu().numpy().astype(np.float64)
    K = solve.fine_kernel(T, cfg["G"], cfg["r_split"], cfg["r_cut"])
    a_t = solve.accel_tile(win, K)[:, bb:bb + t, bb:bb + t, bb:bb + t]
    s0 = tix * t
    got_t = af[:, s0[2]:s0[2] + t, s0[1]:s0[1] + t, s0[0]:s0[0] + t].cpu().numpy()
    assert rel_rms(got_t, a_t) < 1e-5
    # interpolation at the decoded particles of the sub-box's interior cells
    xin = np.concatenate(xs_sample).astype(np.float32)
    inside = np.all((xin >= a) & (xin < b), axis=1)
    xin = xin[inside]
    ag = pm.interpolate(torch.from_numpy(xin).cuda(), ac, af).cpu().numpy()
    fa = af[:, a[2]:b[2] + 1, a[1]:b[1] + 1, a[0]:b[0] + 1].cpu().numpy()
    ca, cb = c0, c0 + k
    fc = ac[:, ca[2]:cb[2] + 1, ca[1]:cb[1] + 1, ca[0]:cb[0] + 1].cpu().numpy()
    ref = mesh.cic_interp(fa, xin.astype(np.float64) - a, 4 * k + 1) + \
        mesh.cic_interp(fc, xin.astype(np.float64) / 4.0 - ca, k + 1)
    assert xin.shape[0] > 1000 and rel_rms(ag, ref) < 1e-6
    del rc, rf, ac, af, fa, fc
    gc.collect()
    torch.cuda.empty_cache()

    # the fused step at full size: status clean, particles conserved, v_max' set
    out = [pm.empty_codes(c.n, esc_cap=c.esc.shape[0]) for c in codes]
    pm.step(codes, out, 1.0, 1.0)
    pm.check()
    for s in range(2):
        cnt = out[s].cnt.to(torch.int64)
        ne = int(out[s].n_esc.item())
        esc = out[s].esc[:ne].cpu().numpy().view(np.uint32)
        tot = int(cnt.sum().item()) - 255 * ne + int(esc[:, 1].astype(np.int64).sum())
        assert tot == counts[s]
        vm = float(out[s].vmax.item())
        assert np.isfinite(vm) and vm > 0
    pm.close()
