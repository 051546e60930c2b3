"""Pins of the constrained (divergence-free) projection of an impressed
magnetic flux density (Section III-C, eq. conB; Tables tab:divblin and
tab:divbsin), against the values the paper prints."""

import json
import os

import numpy as np
import pytest

import workloads
from oracle import geometry, project, topology

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _lin(x):
    return np.stack([x[:, 1], x[:, 0], 0 * x[:, 0]], axis=1)


def _sin(x):
    return np.stack([np.sin(x[:, 1]), np.cos(x[:, 0]), 0 * x[:, 0]], axis=1)


def _box(order):
    gold = json.load(open(GOLDEN))["sinusoidal_field_reconstruction"]
    xyz, tets = workloads.kuhn_box(3, 3, 3, lengths=tuple(gold["box_m"]), jitter=0.1, seed=3)
    t = topology.Topology(xyz, tets, order)
    g, c, vol = geometry.barycentric_maps(t.xyz, t.tets)
    return t, g, c, vol


def test_w3_spans_the_divergence_space():
    """W3 of order p has dim P_{p-1} per tet (Appendix count k(k+1)(k+2)/6)."""
    for p in (1, 2, 3):
        assert len(project.w3_spec(p)) == p * (p + 1) * (p + 2) // 6


@pytest.mark.parametrize("order", [1, 2, 3])
def test_sinusoidal_field_table(order):
    gold = json.load(open(GOLDEN))["sinusoidal_field_reconstruction"]
    t, g, c, vol = _box(order)
    bg = project.project(t, g, vol, _sin, constrained=False)
    bc = project.project(t, g, vol, _sin, constrained=True)
    eg, dg = project.errors(t, g, c, vol, bg, _sin)
    ec, dc = project.errors(t, g, c, vol, bc, _sin)
    m = f"m{order}"
    for got, want in ((eg, gold["error_B_nonconstrained"][m]), (ec, gold["error_B_constrained"][m])):
        assert want / 2.5 < got < want * 2.5
    assert dc < 1e-11                     # Gauss's magnetic law to machine precision
    assert dg > 1e4 * dc                  # the Galerkin projection is not divergence free
    if order > 1:                         # the error falls by more than 10x per order
        t1, g1, c1, vol1 = _box(order - 1)
        b1 = project.project(t1, g1, vol1, _sin, constrained=True)
        assert ec < 0.1 * project.errors(t1, g1, c1, vol1, b1, _sin)[0]


@pytest.mark.parametrize("order", [1, 2])
def test_linear_field_table(order):
    """y x^ + x y^: exact at order >= 2 with and without the constraint; at
    order 1 only the constrained projection is divergence free."""
    t, g, c, vol = _box(order)
    for con in (False, True):
        b = project.project(t, g, vol, _lin, constrained=con)
        err, dv = project.errors(t, g, c, vol, b, _lin)
        if order >= 2:
            assert err < 1e-13 and dv < 1e-11
        elif con:
            assert err > 1e-3 and dv < 1e-11
        else:
            assert err > 1e-3 and dv > 1e-3
