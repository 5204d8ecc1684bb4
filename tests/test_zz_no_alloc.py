"""pm_decompress_noalloc: decompression for callers that may not allocate
device memory (applications that own the device memory budget, or threads
that must not incur cudaMalloc's device-wide synchronisation).  It must give
exactly what pm_decompress gives, call after call, although its scratch is a
fixed array inside the library that every call reuses."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import codec
from synth import make_workload
from tests.helpers import lib_codes_from_oracle

pytestmark = pytest.mark.gpu


def _noalloc(lib, n_fine, vel_bits, dc, stream):
    x = torch.empty((dc.n, 3), dtype=torch.float32, device="cuda")
    v = torch.empty((dc.n, 3), dtype=torch.float32, device="cuda")
    s = dc.struct()
    rc = lib.pm_decompress_noalloc(n_fine, 4, vel_bits, ctypes.byref(s), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    return rc, x, v


@pytest.mark.parametrize("vel_bits", [16, 8])
def test_noalloc_matches_pm_decompress_twice(vel_bits):
    from paper_1611_01545_gb300 import PM, _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    w = make_workload("two_level128_t96", n_cdm=24, n_nu=61)
    pm = PM(dict(w.config(), vel_bits=vel_bits))
    for call in range(2):                      # the shared scratch keeps the previous call's contents
        for s in range(2):
            ref = codec.compress(w.x[s], w.v[s], w.n_fine, w.n_fine // 4, vel_bits)
            dc = lib_codes_from_oracle(ref)
            x0, v0 = pm.decompress(s, dc)
            pm.check()
            rc, x1, v1 = _noalloc(lib, w.n_fine, vel_bits, dc, stream)
            assert rc == 0, (call, s, rc)
            # the codec is bit-exact, so the two entry points must agree bit for bit
            assert torch.equal(x0, x1) and torch.equal(v0, v1)
    pm.close()


def test_noalloc_rejects_oversized_mesh_and_reports_corruption():
    from paper_1611_01545_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    x = (rng.random((500, 3)) * 32).astype(np.float32)
    c = codec.compress(x, rng.standard_normal((500, 3)).astype(np.float32), 32, 8, 16)
    dc = lib_codes_from_oracle(c)
    rc, _, _ = _noalloc(lib, 512, 16, dc, stream)      # 128^3 compression cells > 64^3
    assert rc == 1
    bad = lib_codes_from_oracle(c)
    bad.cnt[int(torch.nonzero(bad.cnt < 200)[0])] += 1
    rc, _, _ = _noalloc(lib, 32, 16, bad, stream)
    assert rc == 4
    rc, x1, _ = _noalloc(lib, 32, 16, dc, stream)       # a clean call after a corrupt one
    assert rc == 0
    np.testing.assert_array_equal(x1.cpu().numpy(), codec.decompress(c, 32)[0])


def test_noalloc_allocates_nothing_and_takes_the_largest_mesh():
    """At the size limit (n_fine 256, cmp_ratio 4: exactly 64^3 compression
    cells) the call succeeds, agrees with pm_decompress bit for bit, and
    repeated calls leave the device's free memory unchanged."""
    from paper_1611_01545_gb300 import PM, _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(6)
    n = 256
    x = (rng.random((40000, 3)) * n).astype(np.float32)
    c = codec.compress(x, rng.standard_normal((40000, 3)).astype(np.float32), n, n // 4, 16)
    dc = lib_codes_from_oracle(c)
    pm = PM(dict(n_fine=n, coarse_ratio=4, tile=64, buffer=16, cmp_ratio=4, vel_bits=16, G=1.0, mass=(1.0, 1.0),
                 count=(c.n, 0), r_split=14.0 / 4.5, r_cut=14.0))
    x0, v0 = pm.decompress(0, dc)
    pm.check()
    outs = [(torch.empty((c.n, 3), dtype=torch.float32, device="cuda"),
             torch.empty((c.n, 3), dtype=torch.float32, device="cuda")) for _ in range(3)]
    s = dc.struct()

    def call(xo, vo):
        return lib.pm_decompress_noalloc(n, 4, 16, ctypes.byref(s), ctypes.c_void_p(xo.data_ptr()),
                                         ctypes.c_void_p(vo.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert call(*outs[0]) == 0                      # warm-up: device address looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for xo, vo in outs[1:]:
        assert call(xo, vo) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for xo, vo in outs:
        assert torch.equal(xo, x0) and torch.equal(vo, v0)
    pm.close()
