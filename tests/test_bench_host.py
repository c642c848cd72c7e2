"""Host-side logic of bench.py, without a GPU: the algorithmic operation
counts behind the roofline (closed forms of the LU and solve costs), their
FP64/FP32 split, and the rule that a DRAM-traffic figure only applies to the
kernel sources it was measured on."""
import sys

import numpy as np

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1607_03884_gb300 import synth  # noqa: E402


def test_linear_algebra_counts_are_the_closed_forms():
    mech = synth.make_mechanism("h2")
    ops = bench.op_model(mech)
    N = mech.ns
    # real LU 2N^3/3 + complex LU 8N^3/3 (+ building E1, E2): 7.3 kflop at N = 13
    assert abs(ops["lu"] - (10.0 / 3.0 * N ** 3 + 3 * N * N)) < 1e-9
    assert 7300 < ops["lu"] - 3 * N * N < 7330
    # one real and one complex solve per Newton iteration: 10 N^2 (+ transforms)
    assert ops["sol"] == 10 * N * N + 40 * N
    assert ops["jac"] > ops["rhs"] > 0


def test_fp32_matrices_move_the_linear_algebra_out_of_the_fp64_count():
    ops = {"rhs": 1000.0, "jac": 3000.0, "lu": 7000.0, "sol": 2000.0, "err": 100.0}
    tot = {"nfcn": 10, "njac": 2, "naccpt": 5, "ndec": 3, "nsol": 4}
    f64, f32 = bench.algorithmic_flops(tot, ops, fp32=True)
    assert f64 == 10 * 1000 + 2 * 3000 + 5 * 100
    assert f32 == 3 * 7000 + 4 * 2000
    g64, g32 = bench.algorithmic_flops(tot, ops, fp32=False)
    assert g64 == f64 + f32 and g32 == 0.0


def test_traffic_figure_needs_matching_kernel_sources(monkeypatch):
    import json
    import os
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    key = next(iter(rec["kernels"]))
    per = rec["kernels"][key]["bytes_per_state"]
    monkeypatch.setattr(bench, "kernel_digest", lambda: rec["sources_digest"])
    assert bench.dram_traffic(key, 1000) == per * 1000
    assert bench.dram_traffic("no-such-kernel", 1000) is None
    monkeypatch.setattr(bench, "kernel_digest", lambda: "0" * 16)
    assert bench.dram_traffic(key, 1000) is None


def test_kernel_digest_is_stable_and_covers_the_sources():
    d = bench.kernel_digest()
    assert d == bench.kernel_digest() and len(d) == 16
    assert np.all([c in "0123456789abcdef" for c in d])
