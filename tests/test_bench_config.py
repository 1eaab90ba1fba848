"""Host-side choices of the benchmark (no GPU): the staging mode by M's type,
the device M pool of the headline workload (one batch of distinct matrices, so
that no slot of a batch finds its M in L2), and the roofline's algorithmic
bytes per batch, (32/R_b + 16/NQ) B per element-update."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2105_00027_gb300 import inputs  # noqa: E402


def _args(**kw):
    a = dict(staging="auto", m_pool=0)
    a.update(kw)
    return SimpleNamespace(**a)


def test_staging_follows_the_type_of_M():
    c64 = inputs.workload("c64_w64")
    c36 = inputs.workload("c36_w64")
    assert c64.m_dtype == "c64" and c36.m_dtype == "c128"
    assert bench.staging_of(c64, _args()) == "deferred"
    assert bench.staging_of(c36, _args()) == "eager"
    assert bench.staging_of(c36, _args(staging="deferred")) == "deferred"
    assert bench.staging_of(c64, _args(staging="eager")) == "eager"


def test_headline_pool_is_one_batch_of_distinct_M():
    p = inputs.workload("c64_w64")
    pool = bench.default_pool(p, _args())
    assert pool >= p.batch and pool <= p.R
    assert bench.default_pool(p, _args(m_pool=7)) == 7
    c16 = inputs.workload("c16_w64")
    assert bench.default_pool(c16, _args()) == c16.R


def test_algorithmic_bytes_per_batch():
    p = inputs.workload("c64_w64")
    E, Rb = p.entries, p.batch
    per_update = 32.0 / Rb + 16.0 / p.NQ
    assert abs((32 * E + 16 * p.N * p.N * Rb) - per_update * E * Rb) < 1e-6 * 32 * E
