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
