"""The bench line's roofline arithmetic (host logic, no GPU): for the PDHG
phase of facility location, achieved = the batch's algorithmic bytes per
iteration x iterations / event time, frac = achieved / the measured peak, traffic = the
one-instance DRAM bytes per iteration x the instances; the dominant phase is
the one with the largest event time."""
import importlib.util
import os

import pytest

from paper_2510_27117_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_facility_pdhg_roofline(bench):
    inst = W.facility_location(nf=20, nc=100, idx=1)
    insts = [inst] * 4
    n = inst.n
    nnz = inst.nnz()
    m = inst.m1 + inst.m2
    iters, ms = 50, 10.0
    prof = {"pdhg": (ms, iters), "sample": (2.0, 4), "eval": (1.0, 4), "incumbent": (0.1, 4)}
    peaks = {"hbm_gbs": 6503.4}
    out = bench.roofline("facility", insts, 50, 256, prof, peaks, "measured", 1)
    alg = (16 * nnz + 24 * n + 16 * m) * len(insts)     # the batch's bytes per iteration
    assert out["phase"] == "pdhg" and out["bound"] == "hbm" and out["unit"] == "GB/s"
    assert out["achieved"] == pytest.approx(alg * iters / (ms / 1e3) / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 6503.4)
    per_inst = bench.TRAFFIC_PER_INSTANCE_ITER["facility"][0]
    assert out["traffic"] == pytest.approx(per_inst * 4)
    assert out["us_per_iteration"] == pytest.approx(ms / iters * 1e3)
    assert out["share"] == pytest.approx(ms / (ms + 2.0 + 1.0 + 0.1))


def test_dominant_phase_is_the_longest(bench):
    inst = W.facility_location(nf=20, nc=100, idx=1)
    prof = {"pdhg": (1.0, 50), "sample": (5.0, 4), "eval": (1.0, 4)}
    out = bench.roofline("facility", [inst], 50, 256, prof, {"hbm_gbs": 6503.4}, "measured", 1)
    assert out["phase"] == "sample"
