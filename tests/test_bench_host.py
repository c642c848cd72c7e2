"""Host-side logic of bench.py, without a GPU: the counted operations behind
the roofline (reproduced from oracle/opcount.py, closed forms of the LU and
solve costs), their FP64/FP32 split, and the rule that a DRAM-traffic figure
only applies to the kernel sources it was measured on."""
import sys

import numpy as np

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1607_03884_gb300 import synth  # noqa: E402


def test_committed_counts_are_reproduced_and_used():
    """oracle/flop_counts.json is what oracle/opcount.py counts now, and
    bench.op_model reads it for both named mechanisms."""
    import json
    import os
    from oracle import opcount
    doc = json.load(open(opcount.COUNTS_PATH))
    for kind in ("h2", "ch4"):
        mech = synth.make_mechanism(kind)
        st = synth.make_states(mech, 3, seed=77)
        y = np.concatenate([st.T[None], st.Y[:-1]])
        fresh = opcount.count_mechanism(mech, y, st.P)
        fresh["per_event"] = opcount.per_event(fresh)
        phis = np.stack([opcount.conc_state(mech, st.Y[:, i], st.T[i], st.P[i])
                         for i in range(st.n)], axis=1)
        conc = opcount.count_conc(mech, phis, st.P)
        conc["per_event"] = opcount.per_event(conc)
        fresh["conc"] = conc
        assert doc["mechanisms"][kind] == json.loads(json.dumps(fresh)), kind
        assert bench.op_model(mech) == fresh["per_event"]
        assert bench.op_model(mech, form="conc") == conc["per_event"]
    other = synth.make_mechanism("h2", seed=999)
    assert bench.op_model(other) is None


def test_linear_algebra_counts_are_the_closed_forms():
    """The counted LU and solves equal their closed forms: real LU
    n(n-1)/2 divisions + 2 sum (n-k-1)^2, complex 11 and 8 per complex
    division and multiply-subtract (~2n^3/3 and ~8n^3/3)."""
    from oracle import opcount
    for kind in ("h2", "ch4"):
        rec = opcount.load_counts(synth.make_mechanism(kind))
        cf = rec["closed_forms"]
        for key in ("lu_real", "lu_cplx", "solve_real", "solve_cplx"):
            assert rec[key]["flops"] == cf[key], (kind, key)
            assert rec[key]["transcendentals"] == 0
        N = rec["N"]
        assert abs(cf["lu_real"] - 2 * N ** 3 / 3) < N ** 2
        assert abs(cf["lu_cplx"] - 8 * N ** 3 / 3) < 4 * N ** 2
    assert opcount.closed_forms(13)["lu_real"] + opcount.closed_forms(13)["lu_cplx"] == 7436


def test_fp32_matrices_move_the_linear_algebra_out_of_the_fp64_count():
    ops = {"rhs": 1000.0, "jac": 3000.0, "lu": 7100.0, "lu_linear": 7000.0, "sol": 2100.0,
           "sol_linear": 2000.0, "err": 150.0, "err_linear": 100.0, "step": 40.0,
           "accept": 20.0}
    tot = {"nfcn": 10, "njac": 2, "naccpt": 5, "nrejct": 1, "ndec": 3, "nsol": 4, "nstep": 7}
    g64, g32 = bench.algorithmic_flops(tot, ops, fp32=False)
    assert g32 == 0.0
    assert g64 == 10 * 1000 + 2 * 3000 + 3 * 7100 + 4 * 2100 + 6 * 150 + 7 * 40 + 5 * 20
    f64, f32 = bench.algorithmic_flops(tot, ops, fp32=True)
    assert f32 == 3 * 7000 + 4 * 2000 + 6 * 100 + 2 * 3000
    assert f64 + f32 == g64


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
