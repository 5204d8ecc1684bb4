"""The torch power-spectrum estimator of the compression study
(paper_1611_01545_gb300/analysis.py) against oracle/power.py on CPU
tensors (its CIC fields come from the library's pm_deposit_weights,
checked against the oracle in tests/test_gpu_analysis.py)."""
import numpy as np
import torch

from oracle import power


def test_power_spectrum_matches_oracle():
    from paper_1611_01545_gb300.analysis import power_spectrum
    rng = np.random.default_rng(3)
    for n in (8, 12, 16):
        f = rng.standard_normal((n, n, n))
        js, P, _ = power.power_spectrum(f)
        jt, Pt = power_spectrum(torch.from_numpy(f))
        np.testing.assert_array_equal(jt.numpy(), js)
        np.testing.assert_allclose(Pt.numpy(), P, rtol=1e-10)
