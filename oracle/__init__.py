"""Oracle for the two-species particle-mesh step -- TEST INFRASTRUCTURE ONLY.

A plain, slow, float64 CPU restatement (numpy) of the PM force step that the
paper describes (Emberson et al., "Cosmological neutrino simulations at
extreme scale"): the cell-ordered compression of Sec. 2.4, the CIC density
of Sec. 2.3, the Fourier-space Poisson solve of Eqs. 1-3 with the two-level
coarse/fine split of Sec. 2.1, CIC force interpolation, a kick-drift update
and recompression.

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path and must never be called by the product.

Parity status of each function is stated in its module docstring; every
function here is pinned by a ``-m "not gpu"`` test against closed forms,
invariants, brute force or values fixed by the paper.
"""
from . import codec, fft, mesh, solve, step  # noqa: F401
