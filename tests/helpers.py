"""Test-side conversions between oracle codes (numpy) and library codes (torch)."""
from __future__ import annotations

import numpy as np
import torch

from oracle import codec


def lib_codes_from_oracle(c: codec.Codes, device="cuda", esc_cap=None):
    from paper_1611_01545_gb300 import Codes
    n = c.n
    cap = max(1, c.esc_cell.size if esc_cap is None else esc_cap)
    esc = np.zeros((cap, 2), np.uint32)
    esc[:c.esc_cell.size, 0] = c.esc_cell
    esc[:c.esc_cell.size, 1] = c.esc_count
    pos = np.zeros((n, 4), np.uint8)
    pos[:, :3] = c.pos
    vel = np.zeros((n, 4), np.uint16 if c.vel_bits == 16 else np.uint8)
    vel[:, :3] = c.vel
    if c.vel_bits == 16:
        vel = vel.view(np.int16)
    return Codes(n=n, cnt=torch.from_numpy(c.cnt.copy()).to(device),
                 esc=torch.from_numpy(esc.view(np.int32)).to(device),
                 n_esc=torch.tensor([c.esc_cell.size], dtype=torch.int32, device=device),
                 pos=torch.from_numpy(pos).to(device),
                 vel=torch.from_numpy(np.ascontiguousarray(vel)).to(device),
                 vmax=torch.tensor([float(c.vmax)], dtype=torch.float32, device=device))


def oracle_codes_from_lib(c, n_cmp: int, vel_bits: int) -> codec.Codes:
    ne = int(c.n_esc.cpu().item())
    esc = c.esc.cpu().numpy().view(np.uint32)[:ne]
    vel = c.vel.cpu().numpy()
    vel = vel.view(np.uint16) if vel_bits == 16 else vel.astype(np.uint8)
    pos = c.pos.cpu().numpy()
    assert np.all(pos[:, 3] == 0) and np.all(vel[:, 3] == 0), "pad bytes must be zero"
    return codec.Codes(n_cmp=n_cmp, vel_bits=vel_bits, cnt=c.cnt.cpu().numpy().copy(),
                       esc_cell=esc[:, 0].copy(), esc_count=esc[:, 1].copy(), pos=pos[:, :3].copy(),
                       vel=vel[:, :3].copy(), vmax=np.float32(c.vmax.cpu().item()))


def records(c: codec.Codes) -> np.ndarray:
    """(cell, px, py, pz, vx, vy, vz) rows sorted lexicographically: the multiset of a species' codes."""
    cell = codec.cell_of_particles(c)
    rec = np.concatenate([cell[:, None], c.pos.astype(np.int64), c.vel.astype(np.int64)], axis=1)
    order = np.lexsort(rec.T[::-1])
    return rec[order]


def multiset_overlap(a: np.ndarray, b: np.ndarray) -> int:
    """Number of records common to both multisets (rows of equal width)."""
    def keys(r):
        k = np.zeros(r.shape[0], dtype=object)
        return [tuple(x) for x in r.tolist()]
    from collections import Counter
    ca, cb = Counter(keys(a)), Counter(keys(b))
    return sum(min(v, cb[k]) for k, v in ca.items())


def rel_rms(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2)) / max(np.sqrt(np.mean(b ** 2)), 1e-300))


def cfg_of(w, **kw):
    c = w.config()
    c.update(kw)
    return c


def _record_keys(c: codec.Codes):
    """Per record: absolute position codes P_d = cell_d * 256 + p_d (1/256 of a
    compression cell per unit, so a move across a cell face is one unit) and
    the velocity codes, as tuples."""
    n = c.n_cmp
    cell = codec.cell_of_particles(c)
    cxyz = np.stack([cell % n, (cell // n) % n, cell // (n * n)], axis=1)
    P = cxyz * 256 + c.pos.astype(np.int64)
    return [tuple(r) for r in np.concatenate([P, c.vel.astype(np.int64)], axis=1).tolist()]


def _pair_off(left_a, left_b, period, offsets):
    """Pairs leftover records of a with leftover records of b at the given
    coordinate offsets (position coordinates periodic); returns the count."""
    paired = 0
    for key, cnt in list(left_a.items()):
        for _ in range(cnt):
            hit = None
            for off in offsets:
                k2 = list(key)
                for j, dlt in off:
                    k2[j] += dlt
                    if j < 3:
                        k2[j] %= period
                k2 = tuple(k2)
                if left_b.get(k2, 0) > 0:
                    hit = k2
                    break
            if hit is None:
                continue
            left_b[hit] -= 1
            if left_b[hit] == 0:
                del left_b[hit]
            left_a[key] -= 1
            paired += 1
    return paired


_ONE = [((j, d),) for j in range(6) for d in (-1, 1)]
_TWO = [((i, a), (j, b)) for i in range(6) for j in range(i + 1, 6) for a in (-1, 1) for b in (-1, 1)]


def code_pairing(got: codec.Codes, ref: codec.Codes, detail: bool = False):
    """Compare one species' codes with the oracle's as multisets of records.

    Records found in only one of the two must pair one to one with a record of
    the other that differs by one quantisation step of one coordinate: one
    velocity code by +-1, or one position coordinate by +-1/256 of a
    compression cell, counted across cell faces (byte 255 of a cell beside
    byte 0 of the next, periodic).  Those are the particles whose float32
    update lands on the other side of a bin edge than the float64 one.  The
    records left after that may pair at one step in each of two coordinates
    (a particle near an edge in two of its six coordinates at once).
    Returns (exact, paired_one, paired_two, unpaired_got, unpaired_ref); with
    detail=True also the unpaired records of each side as (P_x, P_y, P_z,
    V_x, V_y, V_z)."""
    from collections import Counter
    period = got.n_cmp * 256
    ka, kb = Counter(_record_keys(got)), Counter(_record_keys(ref))
    exact = sum(min(v, kb[k]) for k, v in ka.items())
    left_a = ka - kb
    left_b = kb - ka
    one = _pair_off(left_a, left_b, period, _ONE)
    two = _pair_off(left_a, left_b, period, _TWO)
    ua = sum(v for v in left_a.values() if v > 0)
    ub = sum(v for v in left_b.values() if v > 0)
    if detail:
        return (exact, one, two, ua, ub, [k for k, v in left_a.items() if v > 0],
                [k for k, v in left_b.items() if v > 0])
    return exact, one, two, ua, ub


STRADDLE_MAX = 0.02   # records allowed to sit one quantisation step from the oracle's
DOUBLE_MAX = 1e-4     # ... and one step in each of two coordinates (plus one record)


def assert_codes_match(got: codec.Codes, ref: codec.Codes, label: str = "", max_frac: float = STRADDLE_MAX):
    """Same particle count and cell counts' total; every record equal to an
    oracle record or one quantisation step from one (code_pairing), those at
    most max_frac of the records, and at most 1 + 1e-4 n of them one step off
    in two coordinates.  Prints the fractions; returns the one-step fraction."""
    assert got.n == ref.n and got.counts().sum() == ref.counts().sum() == ref.n
    exact, one, two, ua, ub, la, lb = code_pairing(got, ref, detail=True)
    frac = (one + two) / max(ref.n, 1)
    print(f"{label}: {exact} records equal, {one} one step apart, {two} one step apart in two coordinates "
          f"({frac:.4%}), {ua}/{ub} unpaired")
    assert ua == 0 and ub == 0, (f"{label}: {ua} GPU / {ub} oracle records have no partner within one step: "
                                 f"GPU {la[:5]} oracle {lb[:5]}")
    assert two <= 1 + DOUBLE_MAX * ref.n, f"{label}: {two} records one step off in two coordinates"
    assert frac <= max_frac, f"{label}: {frac:.4%} of records one step apart"
    return frac


def device_records_equal(a, b, n_cmp: int) -> bool:
    """Two species' library codes (device tensors) hold the same multiset of
    records per cell: equal count bytes and escape entries, and equal records
    after sorting both streams by (cell, position bytes, velocity codes) on
    the device (for particle counts where host-side sorting is slow)."""
    import torch
    if a.n != b.n or not torch.equal(a.cnt, b.cnt) or not torch.equal(a.n_esc, b.n_esc):
        return False
    ne = int(a.n_esc.item())
    if ne and not torch.equal(a.esc[:ne], b.esc[:ne]):
        return False
    counts = a.cnt.to(torch.int64)
    if ne:
        e = a.esc[:ne].to(torch.int64) & 0xFFFFFFFF
        counts[e[:, 0]] = e[:, 1]
    cell = torch.repeat_interleave(torch.arange(n_cmp ** 3, device=a.cnt.device), counts)

    def keys(c):
        p = c.pos.to(torch.int64)
        hi = (cell << 24) | p[:, 0] | (p[:, 1] << 8) | (p[:, 2] << 16)
        v = c.vel.to(torch.int64) & (0xFFFF if c.vel.dtype == torch.int16 else 0xFF)
        sh = 16 if c.vel.dtype == torch.int16 else 8
        lo = v[:, 0] | (v[:, 1] << sh) | (v[:, 2] << (2 * sh))
        i1 = torch.sort(lo, stable=True).indices
        i2 = torch.sort(hi[i1], stable=True).indices
        o = i1[i2]
        return hi[o], lo[o]
    ha, la = keys(a)
    hb, lb = keys(b)
    return bool(torch.equal(ha, hb) and torch.equal(la, lb))
