"""The committed golden fixture (written by tests/golden/make_golden.py from the
oracle only) is reproduced by the oracle, and by the CUDA path on the GPU."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config1_4x4.json")))


def _arr(key):
    a = np.array(G[key])
    return (a[:, 0] + 1j * a[:, 1]).reshape(len(G["cols"]), len(G["sites"]), 4, 3)


def _setup():
    dims = tuple(G["dims"])
    U = inputs.random_su3_field(dims, G["eps"], G["seed"])
    return dims, U


def test_oracle_reproduces_golden():
    dims, U = _setup()
    op = oracle.Operator(dims, U, G["kappa"], G["csw"])
    eta = inputs.point_sources(dims, tuple(G["x_src"]))
    fact = oracle.factorized_propagator(op, oracle.Split(tuple(G["gamma"]), tuple(G["gamma_star"])), eta)
    s, c = G["sites"], G["cols"]
    assert np.abs(fact[c][:, s] - _arr("fact")).max() < 1e-12
    # the identity full = fact + corr holds in the stored values
    assert np.abs(_arr("full") - _arr("fact") - _arr("corr")).max() < 1e-15


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [64, 32])
def test_cuda_reproduces_golden(prec):
    import torch

    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims, U = _setup()
    lat = lqcd.Lattice(dims, G["bc"])
    lat.set_gauge(U, G["kappa"], G["csw"])
    fact, corr, st = lat.factorized_propagator(tuple(G["gamma"]), tuple(G["gamma_star"]), tuple(G["x_src"]),
                                               params=lqcd.SolverParams(tol=1e-12 if prec == 64 else 1e-10,
                                                                        precision=prec))
    torch.cuda.synchronize()
    s, c = G["sites"], G["cols"]
    scale = np.abs(_arr("full")).max()
    assert np.abs(fact.cpu().numpy()[c][:, s] - _arr("fact")).max() <= 2e-9 * scale
    assert np.abs(corr.cpu().numpy()[c][:, s] - _arr("corr")).max() <= 2e-9 * scale
