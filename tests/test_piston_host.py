"""The library's differential-piston operator, formed on the host (letkf_piston_operator: FP64
Cholesky of the domains' normal matrix plus the no-added-piston projection), against the oracle's
minimum-norm least squares (oracle.piston), with no GPU: the whole-pupil workloads and a pupil of
two separate islands (two groups of domains, each with its own free constant); and the device
bytes the mode adds."""

import os
import sys

import numpy as np
import pytest

from oracle import geometry, piston
from oracle.fried import fried_matrix
from paper_1310_5954_gb300 import _lib
from paper_1310_5954_gb300 import build as builder
from paper_1310_5954_gb300.letkf import footprint, make_params

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _islands():
    sv = np.zeros((12, 12), dtype=bool)
    sv[0:4, 0:5] = True
    sv[7:12, 6:12] = True
    return sv


def _case(name):
    if name == "islands":
        sv = _islands()
        g = geometry.make_geometry(12, 0.0, sub_valid=sv)
        doms = geometry.make_domains(g, 2, 1)
        kw = dict(n_sub=12, m=20, ar1_a=0.99, sigma=0.1, dom_sub=2, halo=1, sub_valid=sv)
        return g, doms, kw
    from _gpu_common import model
    w, g, doms, L, Ls = model(name)
    kw = dict(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
              obstruction=w.obstruction)
    return g, doms, kw


@pytest.mark.parametrize("name", ["tiny-8x8", "vlt-40x40", "elt-80x80", "islands"])
def test_operator_matches_oracle_least_squares(name):
    g, doms, kw = _case(name)
    p, keep = make_params(**kw, piston="in_loop")
    K = _lib.letkf_piston_operator(p)
    tab = _lib.letkf_domain_tables(p)
    assert K.shape == (len(doms), len(doms))
    for d, dom in enumerate(doms):    # the same domain numbering on both sides
        assert np.array_equal(np.sort(tab["own"][tab["own_off"][d]:tab["own_off"][d + 1]]), dom.owned_act)
    D = fried_matrix(g)
    P = piston.ownership(g, doms)
    rng = np.random.default_rng(17)
    for _ in range(3):
        x = rng.standard_normal(g.n_act) * 3.0
        y = rng.standard_normal(2 * g.n_subv)
        delta = K @ ((D @ P).T @ (y - D @ x))
        ref = piston.differential_pistons(x, y, g, doms)
        assert np.abs(delta - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    if name == "islands":
        assert len(np.unique(piston.domain_groups(g, doms))) == 2


def test_footprint_of_the_mode():
    g, doms, kw = _case("tiny-8x8")
    base = dict(kw, precision="fp32", path="fused", q_white=0.1)
    f0 = footprint(**base)
    f1 = footprint(**base, piston="output")
    assert footprint(**base, piston="in_loop") == f1
    # one 32-byte entry per (domain, subaperture) pair with corners in more than one domain
    owner = np.argmax(piston.ownership(g, doms), axis=1)
    D = fried_matrix(g)
    n_ent = 0
    for k in range(g.n_subv):
        cols = np.nonzero(D[k])[0]
        own = set(owner[cols])
        if len(own) > 1:
            n_ent += len(own)
    nd = len(doms)
    assert f1 - f0 == 32 * n_ent + 4 * (nd + 1) + 4 * (nd * nd + nd + g.n_act)
