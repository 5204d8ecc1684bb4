"""Compression-accuracy study (Sec. 2.4) on the small two-level set with the
paper's 16-bit velocity codes: ten compressed restarts and a single
compression keep the CDM density power within 1% up to k_Nyq/2 and the
velocity power within 1% up to k_Nyq/3, and the neutrino density power
within 1% below the shot-noise scale -- the sub-percent agreement the paper
reports for its own runs."""
import pytest

pytestmark = pytest.mark.gpu


def test_compressed_restarts_keep_power_spectra():
    from paper_1611_01545_gb300.analysis import compression_study, summary
    r = compression_study("two_level64", steps=22, restarts=10, c=0.25, vel_bits=16)
    assert r["restarts"] == 10
    s = summary(r)
    for arm in ("restarts", "single"):
        assert s["cdm"][arm]["density_to_nyq2"] < 0.01, s
        assert s["cdm"][arm]["velocity_to_nyq3"] < 0.01, s
        assert s["nu"][arm]["density_below_k_noise"] < 0.01, s
