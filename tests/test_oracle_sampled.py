"""The oracle's parallel sampled-row driver returns exactly what the oracle
itself computes row by row (F rows of Eq. FF-def, point-sun insolation)."""
import numpy as np

import oracle
import synth
from oracle import sampled


def test_sampled_rows_equal_the_oracle():
    v, f = synth.fbm_dem_mesh(n=24, spacing=5.0, seed=2, crater_diameter=None)
    om = oracle.mesh(v, f)
    rows = np.sort(np.random.default_rng(7).choice(om.n, 37, replace=False))
    dirs = synth.sun_directions(5, 12.0)
    with sampled.SampledOracle(v, f, rows, workers=2, chunk=4) as so:
        ip, ix, dv = so.F_rows_sparse()
        Es = so.insolation_rows(dirs, 1365.0)
    Fr = oracle.F_rows(om, rows)
    dense = np.zeros_like(Fr)
    for r in range(rows.size):
        dense[r, ix[ip[r]:ip[r + 1]]] = dv[ip[r]:ip[r + 1]]
    assert np.array_equal(dense, Fr)
    assert np.array_equal(Es, oracle.insolation(om, dirs, 1365.0)[rows])
    X = np.random.default_rng(1).uniform(size=(om.n, 3))
    assert np.allclose(sampled.csr_matmul(ip, ix, dv, X), Fr @ X, rtol=1e-13, atol=0)
