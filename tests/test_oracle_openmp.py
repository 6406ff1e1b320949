"""The OpenMP build of the oracle (the timed CPU baseline on all host cores) computes the same
bits as the plain build: its loops share out iterations that write disjoint results, and every
sum keeps the plain build's order. No GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1912_12059_gb300 import inputs


@pytest.mark.parametrize("dim,ne,N", [(1, (33,), 3), (2, (9, 7), 4), (3, (5, 4, 6), 3)])
@pytest.mark.parametrize("flux", [O.FLUX_LF, O.FLUX_HLLC])
def test_openmp_build_is_bit_identical(dim, ne, N, flux):
    prm = dict(T=0.85, kappa=1e-3, alpha=1e3, beta=1e-3, mu=2e-2, flux=flux)
    lo, hi = [0.0] * dim, [1.0, 0.8, 1.3][:dim]
    plain = O.Oracle(dim, ne, lo, hi, N, **prm)
    omp = O.Oracle(dim, ne, lo, hi, N, parallel=True, **prm)
    U = inputs.random_state(plain.shape, seed=50 + dim)
    assert np.array_equal(plain.lift(U), omp.lift(U))
    assert np.array_equal(plain.rhs(U), omp.rhs(U))
    dt = plain.timestep(U, 0.5)
    assert omp.timestep(U, 0.5) == dt
    assert np.array_equal(plain.step(U, dt, 3), omp.step(U, dt, 3))
    assert plain.diagnostics(U) == omp.diagnostics(U)


def test_openmp_build_uses_threads_and_reports_errors():
    assert O.threads(parallel=False) == 1
    assert O.threads(parallel=True) >= 1
    o = O.Oracle(2, (4, 4), (0, 0), (1, 1), 3, parallel=True)
    U = inputs.random_state(o.shape, seed=9)
    U[0, 5, 3] = 3.5  # beyond the co-volume limit: the same error as the plain build
    with pytest.raises(O.OracleError):
        o.rhs(U)
