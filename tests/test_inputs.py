"""Seeded synthetic inputs: the vertex-configuration recipe."""
import numpy as np


def test_vertex_config_recipe():
    from paper_2105_00027_gb300 import inputs
    p = inputs.workload("c36_w64")
    assert inputs.vertices_per_spin(p) == 1440
    n_up, n_dn, tau, site, Mt = inputs.vertex_config(p, 3)
    assert n_up == n_dn and abs(n_up - 1440) <= 144
    assert tau.shape == (2 * n_up,) and site.dtype == np.int32 and Mt.shape == (2 * n_up * n_up,)
    assert (tau >= 0).all() and (tau < p.beta).all() and (site >= 0).all() and (site < p.Nc).all()
    assert np.array_equal(tau[:n_up], tau[n_up:]) and np.array_equal(site[:n_up], site[n_up:])
    up = Mt[:n_up * n_up].reshape(n_up, n_up)
    assert 0.4 < np.diag(up).mean() < 1.6
    # reproducible per measurement, independent across measurements
    again = inputs.vertex_config(p, 3)
    assert all(np.array_equal(a, b) for a, b in zip(again[2:], (tau, site, Mt)))
    other = inputs.vertex_config(p, 4, n=10, jitter=False, shared=False)
    assert other[0] == 10 and other[1] == 10 and not np.array_equal(other[2][:10], other[2][10:])
