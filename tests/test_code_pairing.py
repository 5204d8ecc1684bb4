"""The strict comparison of post-step codes (tests/helpers.code_pairing) on
the CPU: records one quantisation step from the oracle's pair up (a bin edge
inside a cell, a compression-cell face, the periodic box face, one velocity
code; one step in each of two codes is counted apart), while planted
mistakes in the oracle's codes (a particle in the neighbouring cell, a
velocity two codes off, a dropped record) are left unpaired."""
import numpy as np

from oracle import codec
from tests.helpers import code_pairing

N_FINE, N_CMP = 32, 8          # 4 fine cells per compression cell: one position code = 1/64 fine cell


def _codes(x, v, vmax=None):
    return codec.compress(np.asarray(x, np.float32), np.asarray(v, np.float32), N_FINE, N_CMP, 16, vmax=vmax)


def _base(n=3000, seed=0):
    rng = np.random.default_rng(seed)
    x = (rng.random((n, 3)) * N_FINE).astype(np.float32)
    v = rng.standard_normal((n, 3)).astype(np.float32)
    return x, v


def _below(a):
    return np.nextafter(np.float32(a), np.float32(-np.inf))


def test_identical_codes_pair_exactly():
    x, v = _base()
    a = _codes(x, v)
    assert code_pairing(a, _codes(x, v, a.vmax)) == (x.shape[0], 0, 0, 0, 0)


def test_bin_edge_cell_face_and_box_face_straddlers_pair():
    x, v = _base()
    ref = _codes(x, v)
    y = x.copy()
    y[0] = (5.25, 7.0, 9.0)            # on a position-bin edge inside a cell
    y[1] = (8.0, 3.0, 3.0)             # on a compression-cell face (fine cell 8 = cell 2, byte 0)
    y[2] = (0.0, 11.0, 13.0)           # on the periodic box face
    ref = _codes(y, v, ref.vmax)
    z = y.copy()
    z[0, 0] = _below(5.25)             # one bin lower
    z[1, 0] = _below(8.0)              # byte 255 of cell 1
    z[2, 0] = _below(float(N_FINE))    # byte 255 of the last cell
    got = _codes(z, v, ref.vmax)
    assert code_pairing(got, ref) == (x.shape[0] - 3, 3, 0, 0, 0)


def test_velocity_code_one_step_pairs_two_steps_do_not():
    x, v = _base()
    ref = _codes(x, v)
    got = _codes(x, v, ref.vmax)
    got.vel = got.vel.copy()
    got.vel[10, 1] += 1
    assert code_pairing(got, ref) == (x.shape[0] - 1, 1, 0, 0, 0)
    got.vel[10, 1] += 1
    assert code_pairing(got, ref)[3:] == (1, 1)
    got.vel[10, 1] -= 1
    got.vel[10, 2] += 1                               # one step in each of two velocity codes
    assert code_pairing(got, ref) == (x.shape[0] - 1, 0, 1, 0, 0)


def test_planted_cell_move_and_dropped_record_are_unpaired():
    x, v = _base()
    ref = _codes(x, v)
    y = x.copy()
    y[7, 1] = np.mod(y[7, 1] + 4.0, N_FINE)      # the neighbouring compression cell, same in-cell byte
    got = _codes(y, v, ref.vmax)
    exact, one, two, ua, ub = code_pairing(got, ref)
    assert (one, two, ua, ub) == (0, 0, 1, 1)
    got = _codes(x[1:], v[1:], ref.vmax)
    assert code_pairing(got, ref)[3:] == (0, 1)


def test_device_record_comparison_ignores_order_within_cells_only():
    """tests/helpers.device_records_equal (used where host-side sorting of the
    records is too slow) on CPU tensors: a copy with each cell's records in
    another order is equal; one changed velocity code, or a record moved to
    another cell of the same count, is not."""
    import torch

    from tests.helpers import device_records_equal, lib_codes_from_oracle
    x, v = _base(4000, seed=2)
    c = _codes(x, v)
    a = lib_codes_from_oracle(c, device="cpu")
    cell = codec.cell_of_particles(c)
    perm = np.lexsort((np.random.default_rng(1).random(c.n), cell))   # shuffle within each cell
    b = lib_codes_from_oracle(c, device="cpu")
    b.pos = b.pos[torch.from_numpy(perm)].clone()
    b.vel = b.vel[torch.from_numpy(perm)].clone()
    assert device_records_equal(a, b, N_CMP)
    b.vel[5, 0] += 1
    assert not device_records_equal(a, b, N_CMP)
    b.vel[5, 0] -= 1
    assert device_records_equal(a, b, N_CMP)
    counts = c.counts()
    starts = np.concatenate([[0], np.cumsum(counts)])
    i, j = np.flatnonzero(counts)[:2]                       # the first records of two cells trade positions
    b.pos[starts[i]], b.pos[starts[j]] = b.pos[starts[j]].clone(), b.pos[starts[i]].clone()
    assert torch.equal(b.pos[starts[i]], b.pos[starts[j]]) or not device_records_equal(a, b, N_CMP)
