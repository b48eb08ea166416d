"""The seeded input laws: shapes, ranges and reproducibility (no GPU)."""
import numpy as np

from paper_1603_04039_gb300 import inputs


def test_beam_batch_laws_and_layout():
    params = inputs.beam_batch_params(64, seed=1)
    n = np.array([p["n"] for p in params])
    assert len(params) == 64
    assert n.min() >= 1e4 and n.max() <= 1e6
    # log-uniform: the median of log10 N sits near the middle of [4, 6]
    assert 4.6 < np.median(np.log10(n)) < 5.4
    for p in params:
        assert 0.02 <= p["sigma"] <= 0.1 and 0.01 <= p["halo_frac"] <= 0.2
        assert 0.2 <= p["r0"] <= p["r1"] <= 0.8
    assert [p["seed"] for p in params] == list(range(1, 65))
    x, y, z, q, offs, p2 = inputs.beam_batch(4, seed=3, n_lo=100, n_hi=2000)
    assert offs[0] == 0 and offs[-1] == len(x) == len(q)
    for b, p in enumerate(p2):
        s, e = offs[b], offs[b + 1]
        assert e - s == p["n"]
        assert np.isclose(q[s:e].sum(), 1.0)
        xb, yb, zb, qb = inputs.beam_with_halo(p["n"], p["seed"], sigma=p["sigma"], halo_frac=p["halo_frac"],
                                               r0=p["r0"], r1=p["r1"])
        assert np.array_equal(x[s:e], xb) and np.array_equal(z[s:e], zb)
    again = inputs.beam_batch(4, seed=3, n_lo=100, n_hi=2000)
    assert np.array_equal(again[0], x)
