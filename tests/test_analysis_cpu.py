"""The torch estimators of the compression study (paper_1611_01545_gb300/
analysis.py) against the oracle on CPU tensors: CIC field against
oracle/mesh.py, power spectrum against oracle/power.py."""
import numpy as np
import torch

from oracle import mesh, power


def test_power_spectrum_matches_oracle():
    from paper_1611_01545_gb300.analysis import power_spectrum
    rng = np.random.default_rng(3)
    for n in (8, 12, 16):
        f = rng.standard_normal((n, n, n))
        js, P, _ = power.power_spectrum(f)
        jt, Pt = power_spectrum(torch.from_numpy(f))
        np.testing.assert_array_equal(jt.numpy(), js)
        np.testing.assert_allclose(Pt.numpy(), P, rtol=1e-10)


def test_cic_field_matches_oracle():
    from paper_1611_01545_gb300.analysis import cic_field
    rng = np.random.default_rng(4)
    n = 10
    x = rng.random((500, 3)) * n
    w = rng.standard_normal(500)
    got = cic_field(torch.from_numpy(x), torch.from_numpy(w), n)[0].numpy()
    np.testing.assert_allclose(got, mesh.cic_deposit(x, w, n), rtol=1e-12, atol=1e-12)
