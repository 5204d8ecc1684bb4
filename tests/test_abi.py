"""Host-only checks of the C ABI: libpm.so loads without a GPU, exports every
function include/pm.h declares, and its host serializer reproduces the
hand-derived Sec. 2.4 byte streams."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import codec
from tests.golden_codec import load_cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_01545_gb300 import _lib, build
    build.build()
    return _lib.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "pm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_1611_01545_gb300 import _lib
    assert sorted(_lib.EXPORTED) == names


def test_error_strings(lib):
    assert lib.pm_error_string(0) == b"ok"
    assert lib.pm_error_string(4) == b"corrupt compressed stream"


def _host_codes(c: codec.Codes):
    from paper_1611_01545_gb300._lib import pm_codes_t
    keep = {}
    esc = np.zeros((max(1, c.esc_cell.size), 2), np.uint32)
    esc[:c.esc_cell.size, 0] = c.esc_cell
    esc[:c.esc_cell.size, 1] = c.esc_count
    keep["cnt"] = np.ascontiguousarray(c.cnt)
    keep["esc"] = esc
    keep["n_esc"] = np.array([c.esc_cell.size], np.uint32)
    pos = np.zeros((c.n, 4), np.uint8)
    pos[:, :3] = c.pos
    vel = np.zeros((c.n, 4), c.vel.dtype)
    vel[:, :3] = c.vel
    keep["pos"] = pos
    keep["vel"] = vel
    keep["vmax"] = np.array([c.vmax], np.float32)
    s = pm_codes_t(c.n, keep["cnt"].ctypes.data, keep["esc"].ctypes.data, esc.shape[0], keep["n_esc"].ctypes.data,
                   keep["pos"].ctypes.data, keep["vel"].ctypes.data, keep["vmax"].ctypes.data)
    return s, keep


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_host_serializer_matches_golden(lib, case):
    c = codec.compress(case["x"], case["v"], case["n_fine"], case["n_cmp"], case["vel_bits"])
    s, keep = _host_codes(c)
    ln = ctypes.c_size_t()
    assert lib.pm_serialize(ctypes.byref(s), case["n_cmp"], case["vel_bits"], None, 0, ctypes.byref(ln)) == 0
    buf = (ctypes.c_uint8 * ln.value)()
    assert lib.pm_serialize(ctypes.byref(s), case["n_cmp"], case["vel_bits"], buf, ln.value, ctypes.byref(ln)) == 0
    assert bytes(buf) == case["hex"]
    # deserialize back into fresh host arrays
    d = codec.Codes(c.n_cmp, c.vel_bits, np.zeros_like(c.cnt), c.esc_cell * 0, c.esc_count * 0,
                    np.zeros_like(c.pos), np.zeros_like(c.vel), np.float32(0))
    s2, keep2 = _host_codes(d)
    src = (ctypes.c_uint8 * len(case["hex"])).from_buffer_copy(case["hex"])
    assert lib.pm_deserialize(src, len(case["hex"]), case["n_cmp"], case["vel_bits"], ctypes.byref(s2)) == 0
    np.testing.assert_array_equal(keep2["pos"][:, :3], c.pos)
    np.testing.assert_array_equal(keep2["vel"][:, :3], c.vel)
    assert np.all(keep2["pos"][:, 3] == 0) and np.all(keep2["vel"][:, 3] == 0)
    np.testing.assert_array_equal(keep2["cnt"], c.cnt)
    assert keep2["vmax"][0] == c.vmax


def test_host_deserializer_rejects_truncation(lib):
    case = load_cases()[0]
    c = codec.compress(case["x"], case["v"], case["n_fine"], case["n_cmp"], case["vel_bits"])
    s, keep = _host_codes(c)
    data = case["hex"][:-3]
    src = (ctypes.c_uint8 * len(data)).from_buffer_copy(data)
    assert lib.pm_deserialize(src, len(data), case["n_cmp"], case["vel_bits"], ctypes.byref(s)) == 4


def test_random_stream_matches_oracle_serializer(lib):
    rng = np.random.default_rng(31)
    x = (rng.random((3000, 3)) * 16).astype(np.float32)
    x[:400] = np.float32(1.25)             # one cell over the 255 escape
    v = rng.standard_normal((3000, 3)).astype(np.float32)
    for vb in (16, 8):
        c = codec.compress(x, v, 16, 4, vb)
        s, keep = _host_codes(c)
        ln = ctypes.c_size_t()
        lib.pm_serialize(ctypes.byref(s), 4, vb, None, 0, ctypes.byref(ln))
        buf = (ctypes.c_uint8 * ln.value)()
        assert lib.pm_serialize(ctypes.byref(s), 4, vb, buf, ln.value, ctypes.byref(ln)) == 0
        assert bytes(buf) == codec.serialize(c)
