"""The workload descriptions in configs/ (one JSON file per workload) are
complete and consistent with the method's rules, and bench.py takes its
parameters from them.

* every curl stencil holds at least twice the monomials of its degree
  (n >= 2 M_m, Sec. 4.1), the wall layer of the 3D cube more than that;
* the hyperviscosity stencils hold 2 M_{2 alpha} + 1 nodes (PHS r^{2 alpha + 1},
  monomials up to 2 alpha; Sec. 5.1);
* the Courant numbers are below the FDTD limit of the dimension (Sec. 3);
* bench.py's parameter tables equal the files.
"""
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = ("c1_cavity", "c2_pulse", "c3_cube", "c4_batched", "c5_adjoint")


def _load(name):
    return json.load(open(os.path.join(ROOT, "configs", name + ".json")))


def _monomials(m, d):
    return math.comb(m + d, d)


@pytest.mark.parametrize("name", NAMES)
def test_config_is_complete_and_follows_the_stencil_rules(name):
    c = _load(name)
    for key in ("name", "workload", "layout", "curl", "hv", "courant", "precision", "steps"):
        assert key in c, key
    d = 3 if name == "c3_cube" else 2
    assert 0 < c["courant"] < 1 / math.sqrt(d)
    alpha = c["hv"]["alpha"]
    if "n" in c["hv"]:
        assert c["hv"]["n"] == 2 * _monomials(2 * alpha, d) + 1
    cu = c["curl"]
    if isinstance(cu.get("poly_m"), int):
        assert cu["n"] >= 2 * _monomials(cu["poly_m"], d)
        assert cu["phs_k"] % 2 == 1
    if "n_wall" in cu:
        assert cu["n_wall"] > cu["n"]
    assert c["precision"] in ("fp32", "fp64")


def test_bench_takes_its_parameters_from_the_files():
    bench = pytest.importorskip("bench")
    c2, c3 = _load("c2_pulse"), _load("c3_cube")
    assert bench.PARAMS == dict(S=c2["courant"], n=c2["curl"]["n"], k=c2["curl"]["phs_k"], m=c2["curl"]["poly_m"],
                                alpha=c2["hv"]["alpha"], c=c2["hv"]["c"], wavelength=c2["wavelength"])
    assert bench.CUBE["n_wall"] == c3["curl"]["n_wall"] and bench.CUBE["c"] == c3["hv"]["c"]
    S, c, nodes, stencil = bench.cavity_setup()
    c1 = _load("c1_cavity")
    assert (S, c) == (c1["courant"], c1["hv"]["c"]) and nodes.n == math.prod(c1["nodes"]["shape"])
    P = bench._adjoint_problem(20)
    c5 = _load("c5_adjoint")
    assert P["stencil"] == (c5["curl"]["n"], c5["curl"]["phs_k"], c5["curl"]["poly_m"], c5["hv"]["n"],
                            c5["hv"]["alpha"])
