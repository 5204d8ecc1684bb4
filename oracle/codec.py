"""Oracle codec: the cell-ordered phase-space compression of Sec. 2.4.

What the paper fixes (Sec. 2.4):
  * particles are binned on a cubic mesh of n_g^3 cells (the long-range mesh)
    and written cell by cell in an ordered fashion;
  * per cell, a 1-byte unsigned count; a count of 255 or more is written as
    255 followed by the real count as a 4-byte integer (footnote);
  * per particle, the position as three unsigned bytes: the digitised offset
    from the cell's local origin, i.e. a precision of (cell width)/256;
  * per particle, the velocity as three 2-byte indices into 2^16 equal bins
    over [-v_max, v_max], with v_max the largest absolute particle velocity,
    kept per species and stored in the file header;
  * species go to separate streams; nothing else (no IDs) is stored.

Readings where the paper is silent (each also listed in the design notes):
  * cells are ordered with x fastest: c = ix + n (iy + n iz);
  * a particle record is px, py, pz (u8) then vx, vy, vz (u16 little-endian);
  * positions decode at bin centres, offset (q + 1/2)/256 of a cell;
  * v_max is the maximum over particles and components of |v_d|;
  * velocity code q = floor(v * s + 2^(b-1)), s = 2^(b-1)/v_max, clamped to
    [0, 2^b - 1], evaluated in IEEE float32 with one rounding per operation
    (the codec is a bit-level definition, so the oracle mirrors float32);
    decode ((q - 2^(b-1)) + 1/2) * (v_max / 2^(b-1)); v_max = 0 gives q =
    2^(b-1) and decodes to 0;
  * b = 16 is the paper's width; b = 8 is the reduced-precision option that
    the paper mentions for the memory-light code (end of Sec. 2.4);
  * within a cell the order is the input stream order ("stable"), or, with
    order="canonical", ascending by the code tuple (px,py,pz,vx,vy,vz).

Pins: tests/test_oracle_codec.py (round trip, error bounds, escape path,
golden byte stream tests/golden/codec_stream_small.txt).
"""
from __future__ import annotations

import struct
from dataclasses import dataclass
from typing import Optional

import numpy as np

ESCAPE = 255
HEADER_MAGIC = b"PMNU"
HEADER_FMT = "<4sIIIQfI"  # magic, version, n_cmp, vel_bits, n_particles, vmax, reserved
HEADER_SIZE = struct.calcsize(HEADER_FMT)


@dataclass
class Codes:
    """One species' compressed state, in the in-memory (SoA) layout."""
    n_cmp: int
    vel_bits: int
    cnt: np.ndarray        # uint8 [n_cmp^3]
    esc_cell: np.ndarray   # uint32 [n_esc], ascending
    esc_count: np.ndarray  # uint32 [n_esc], >= 255
    pos: np.ndarray        # uint8 [n, 3]
    vel: np.ndarray        # uint16 or uint8 [n, 3]
    vmax: np.float32

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def counts(self) -> np.ndarray:
        """Per-cell particle counts (int64), resolving the 255 escape."""
        c = self.cnt.astype(np.int64)
        if self.esc_cell.size:
            if np.any(self.cnt[self.esc_cell] != ESCAPE) or np.any(self.esc_count < ESCAPE):
                raise ValueError("corrupt escape list")
            c[self.esc_cell.astype(np.int64)] = self.esc_count
        if np.count_nonzero(self.cnt == ESCAPE) != self.esc_cell.size:
            raise ValueError("escape byte without escape entry")
        if self.esc_cell.size > 1 and np.any(np.diff(self.esc_cell.astype(np.int64)) <= 0):
            raise ValueError("escape list not ascending")
        return c


def velocity_encode(v: np.ndarray, vmax: np.float32, bits: int) -> np.ndarray:
    half = np.float32(2 ** (bits - 1))
    top = 2 ** bits - 1
    v = np.asarray(v, dtype=np.float32)
    if vmax == 0:
        return np.full(v.shape, int(half), dtype=np.int64)
    s = np.float32(half / np.float32(vmax))           # one IEEE float32 division
    t = (v * s).astype(np.float32)                    # rounded product
    t = (t + half).astype(np.float32)                 # rounded sum
    return np.clip(np.floor(t).astype(np.int64), 0, top)


def velocity_decode(q: np.ndarray, vmax: np.float32, bits: int) -> np.ndarray:
    half = 2 ** (bits - 1)
    step = np.float32(np.float32(vmax) * np.float32(1.0 / half))   # exact power-of-two scaling
    a = (q.astype(np.int64) - half).astype(np.float32) + np.float32(0.5)
    return (a * step).astype(np.float32)


def position_encode(x: np.ndarray, n_fine: int, n_cmp: int):
    """Cell coordinates and 8-bit in-cell offsets of float32 positions on [0, n_fine)."""
    x = np.asarray(x, dtype=np.float32)
    if np.any(x < 0) or np.any(x >= np.float32(n_fine)):
        raise ValueError("positions must lie in [0, n_fine)")
    r = n_fine // n_cmp
    u = x.astype(np.float64) / r            # exact: r is a power of two
    c = np.floor(u)
    f = u - c                                # exact
    q = np.minimum(255, np.floor(f * 256.0)).astype(np.int64)
    return c.astype(np.int64), q


def position_decode(cell_xyz: np.ndarray, q: np.ndarray, n_fine: int, n_cmp: int) -> np.ndarray:
    r = n_fine // n_cmp
    x = (cell_xyz.astype(np.float64) * 256.0 + q.astype(np.float64) + 0.5) * (r / 256.0)
    return x.astype(np.float32)               # exact: a dyadic with few bits


def compress(x, v, n_fine: int, n_cmp: int, vel_bits: int = 16, vmax: Optional[float] = None,
             order: str = "stable") -> Codes:
    """Compress float32 positions/velocities of ONE species (Sec. 2.4)."""
    if vel_bits not in (8, 16):
        raise ValueError("vel_bits must be 8 or 16")
    r = n_fine // n_cmp
    if r * n_cmp != n_fine or r & (r - 1):
        raise ValueError("n_fine / n_cmp must be a power of two")
    x = np.asarray(x, dtype=np.float32).reshape(-1, 3)
    v = np.asarray(v, dtype=np.float32).reshape(-1, 3)
    cxyz, qpos = position_encode(x, n_fine, n_cmp)
    cell = cxyz[:, 0] + n_cmp * (cxyz[:, 1] + n_cmp * cxyz[:, 2])
    if vmax is None:
        vmax = np.float32(np.max(np.abs(v))) if v.size else np.float32(0.0)
    vmax = np.float32(vmax)
    qvel = velocity_encode(v, vmax, vel_bits)
    if order == "stable":
        perm = np.argsort(cell, kind="stable")
    elif order == "canonical":
        keys = (qvel[:, 2], qvel[:, 1], qvel[:, 0], qpos[:, 2], qpos[:, 1], qpos[:, 0], cell)
        perm = np.lexsort(keys)
    else:
        raise ValueError(order)
    counts = np.bincount(cell, minlength=n_cmp ** 3)
    esc = np.nonzero(counts >= ESCAPE)[0]
    vdt = np.uint16 if vel_bits == 16 else np.uint8
    return Codes(n_cmp=n_cmp, vel_bits=vel_bits,
                 cnt=np.minimum(counts, ESCAPE).astype(np.uint8),
                 esc_cell=esc.astype(np.uint32), esc_count=counts[esc].astype(np.uint32),
                 pos=qpos[perm].astype(np.uint8), vel=qvel[perm].astype(vdt), vmax=vmax)


def cell_of_particles(codes: Codes) -> np.ndarray:
    counts = codes.counts()
    if counts.sum() != codes.n:
        raise ValueError("cell counts do not add up to the particle count")
    return np.repeat(np.arange(codes.n_cmp ** 3, dtype=np.int64), counts)


def decompress(codes: Codes, n_fine: int):
    """Decode one species' codes to float32 positions and velocities, in stream order."""
    n = codes.n_cmp
    if not np.isfinite(codes.vmax) or codes.vmax < 0:
        raise ValueError("corrupt vmax")
    cell = cell_of_particles(codes)
    cxyz = np.stack([cell % n, (cell // n) % n, cell // (n * n)], axis=1)
    x = position_decode(cxyz, codes.pos.astype(np.int64), n_fine, n)
    v = velocity_decode(codes.vel, codes.vmax, codes.vel_bits)
    return x, v


def canonicalise(codes: Codes) -> Codes:
    """Re-order each cell's records ascending by (px,py,pz,vx,vy,vz)."""
    cell = cell_of_particles(codes)
    p, q = codes.pos.astype(np.int64), codes.vel.astype(np.int64)
    perm = np.lexsort((q[:, 2], q[:, 1], q[:, 0], p[:, 2], p[:, 1], p[:, 0], cell))
    return Codes(codes.n_cmp, codes.vel_bits, codes.cnt.copy(), codes.esc_cell.copy(),
                 codes.esc_count.copy(), codes.pos[perm].copy(), codes.vel[perm].copy(), codes.vmax)


def serialize(codes: Codes) -> bytes:
    """The byte stream of Sec. 2.4 for one species, after a fixed header.

    Header (little-endian): b"PMNU", version 1, n_cmp, vel_bits, particle count
    (u64), v_max (f32), reserved (u32).  Then for each cell in order: the count
    byte, the escaped 4-byte count if the byte is 255, and the cell's records.
    """
    counts = codes.counts()
    out = bytearray(struct.pack(HEADER_FMT, HEADER_MAGIC, 1, codes.n_cmp, codes.vel_bits, codes.n,
                                float(codes.vmax), 0))
    vfmt = "<3H" if codes.vel_bits == 16 else "<3B"
    p = 0
    for c in range(codes.n_cmp ** 3):
        k = int(counts[c])
        if k >= ESCAPE:
            out += bytes([ESCAPE]) + struct.pack("<i", k)
        else:
            out += bytes([k])
        for j in range(p, p + k):
            out += bytes(codes.pos[j].tolist()) + struct.pack(vfmt, *codes.vel[j].tolist())
        p += k
    return bytes(out)


def deserialize(buf: bytes) -> Codes:
    magic, ver, n_cmp, vel_bits, n, vmax, _ = struct.unpack_from(HEADER_FMT, buf, 0)
    if magic != HEADER_MAGIC or ver != 1 or vel_bits not in (8, 16):
        raise ValueError("bad header")
    vb = 2 if vel_bits == 16 else 1
    vfmt = "<3H" if vel_bits == 16 else "<3B"
    off = HEADER_SIZE
    cnt = np.zeros(n_cmp ** 3, np.uint8)
    esc_c, esc_n, pos, vel = [], [], [], []
    for c in range(n_cmp ** 3):
        if off >= len(buf):
            raise ValueError("truncated stream")
        k = buf[off]
        off += 1
        cnt[c] = k
        if k == ESCAPE:
            (k,) = struct.unpack_from("<i", buf, off)
            off += 4
            if k < ESCAPE:
                raise ValueError("bad escaped count")
            esc_c.append(c)
            esc_n.append(k)
        for _ in range(k):
            if off + 3 + 3 * vb > len(buf):
                raise ValueError("truncated stream")
            pos.append(tuple(buf[off:off + 3]))
            vel.append(struct.unpack_from(vfmt, buf, off + 3))
            off += 3 + 3 * vb
    if off != len(buf) or len(pos) != n:
        raise ValueError("stream length disagrees with header")
    vdt = np.uint16 if vel_bits == 16 else np.uint8
    return Codes(n_cmp, vel_bits, cnt, np.array(esc_c, np.uint32), np.array(esc_n, np.uint32),
                 np.array(pos, np.uint8).reshape(-1, 3), np.array(vel, vdt).reshape(-1, 3), np.float32(vmax))
