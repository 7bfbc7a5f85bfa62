"""The benchmark's method options on CPU: every per-workload setting is a field of
the library's lamg_options and of the oracle's options (so the GPU arm, the
CPU baseline and the reference arm run the same method), and command-line flags
override a workload's settings one by one."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402


@pytest.fixture(scope="module")
def L():
    from paper_1108_1310_gb300 import build
    build.build()
    from paper_1108_1310_gb300 import lamg
    return lamg


def _args(**kw):
    keys = ("gamma", "gamma_coarse_max", "elim", "agg_rule", "recomb_finest", "n_coarsest", "mu_adaptive",
            "colour_rule")
    return argparse.Namespace(**{k: kw.get(k) for k in keys})


def test_workload_options_are_method_fields(L):
    lib_fields = {f[0] for f in L.lamg_options._fields_}
    orc_fields = {f[0] for f in oracle.Opts._fields_}
    engine_only = {"sb_work32", "sb_work64", "tail_work32", "tail_work64"}   # launch shapes, no arithmetic
    for name in list(bench.WORKLOADS) + list(bench.BATCHED) + list(bench.ADJOINT):
        opts, _ = bench.method_opts(name, 1 << 20)
        for k in opts:
            assert k in lib_fields, (name, k)
            assert k in orc_fields or k in engine_only, (name, k)


def test_grid_workload_settings_and_overrides():
    opts, adaptive = bench.method_options(_args(), "grid256", 256 ** 3)
    assert adaptive and opts["gamma"] == 1.2 and opts["gamma_coarse_max"] == 1.0 and opts["colour_rule"] == 1
    opts, _ = bench.method_options(_args(gamma=1.5, mu_adaptive=1.1), "grid256", 256 ** 3)
    assert opts["gamma"] == 1.5 and opts["mu_adaptive"] == 1.1 and opts["gamma_coarse_max"] == 1.0
    opts, _ = bench.method_options(_args(), "grid1024_13pt", 1024 ** 2)
    assert opts == {"negative_weights": 1, "mu_adaptive": 1.2}
    # a workload without settings runs the library's defaults
    opts, _ = bench.method_options(_args(), "rgg2m_b64", 2_000_000)
    assert opts == {}
    # lean geometric MG: flat cycles, mu 2, the torus side from n
    opts, adaptive = bench.method_options(_args(), "torus1024_lgmg", 1024 ** 2)
    assert not adaptive and opts == {"lgmg_nx": 1024, "mu_flat": 2.0}
