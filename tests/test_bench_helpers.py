"""bench.py on the CPU: the byte counts behind its roofline, checked
against independent counts (the oracle's face topology and a direct count
of the (receiver, subdomain) pairs), and the JSON line of its reference
arm."""
import numpy as np
import pytest

import sfm_inputs as inputs
from oracle import faces


def _pairs(p):
    """(receiver, subdomain) pairs: a subdomain's closed node box holds a
    node with nonzero trilinear weight of the receiver."""
    out = 0
    boxes = np.array([p.sub_box(s) for s in range(p.nsub)])
    for x in p.rec_xyz:
        nodes, _ = inputs.trilinear_node_weights(x, p.h, p.nx, p.ny, p.nz)
        hit = np.zeros(p.nsub, dtype=bool)
        for i, j, k in nodes:
            hit |= ((boxes[:, 0] <= i) & (i <= boxes[:, 1]) & (boxes[:, 2] <= j) & (j <= boxes[:, 3])
                    & (boxes[:, 4] <= k) & (k <= boxes[:, 5]))
        out += int(hit.sum())
    return out


def test_face_modes_match_the_oracle_topology():
    import bench
    for p in (inputs.config3(), inputs.small_problem(ncell=(12, 8, 8), cuts=(4, 4, 8),
                                                      m_sub=[3, 5, 4, 6, 2, 7])):
        np.testing.assert_array_equal(bench.face_modes(p), faces.Topology(p).mf)


def test_config2_bytes_per_step():
    """Config 2 (512 subdomains, b = 48, k = 16, m = 8, one shot): packed
    coefficients (2k - 1) b(b+1)/2 per subdomain, six m(m+1)/2 face blocks,
    k b numbers per receiver pair, and per shot U and delta read and written
    plus the face data written and read back."""
    import bench
    p = inputs.config2()
    npairs = _pairs(p)
    assert npairs == 2196          # 1024 receivers on the y = 96h cut plane
    rec = bench.receiver_row_numbers(p)
    assert rec == npairs * 16 * 48
    per_sub = 31 * 48 * 49 // 2 + 6 * 8 * 9 // 2 + 4 * 16 * 48 + 2 * 48
    want = (512 * per_sub + rec) * 4
    assert bench.algorithmic_bytes_per_step(p, 1, rec, (4, 4)) == want == 88338432
    assert bench.algorithmic_bytes_per_step(p, 1, rec, (8, 8)) == 2 * want
    # more shots add only the per-shot state
    assert (bench.algorithmic_bytes_per_step(p, 3, rec, (4, 4)) - want) == 2 * 512 * (4 * 16 * 48 + 2 * 48) * 4
    # FP32 factors with a two-float state: only the blocks stay at 4 bytes
    blocks = 512 * 31 * 48 * 49 // 2
    assert bench.algorithmic_bytes_per_step(p, 1, rec, (4, 8)) == 2 * want - 4 * blocks


def test_two_float_panel_roofline_counts_fp32_operations():
    """The two-float panel mode is bound by FP32 issue: its roof counts
    12 FP32 operations per compensated term and (2k - 1) b^2 terms per
    subdomain, shot and time step, against 152 SMs x 128 lanes x the
    clock; the HBM figure rides beside it."""
    import bench
    p = inputs.config3()
    t = {"kernel_ms": 1000.0, "clocks": {"sm_mhz": 2000.0}}
    r = bench.roofline_of(p, "fp32x2p", t, 100, {"hbm_gbs": 7000.0}, "measured", None)
    b = bench.face_modes(p).sum(axis=1)
    k = np.asarray(p.k_sub)
    terms = float(((2 * k - 1) * b * b).sum()) * p.nshots
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["two_float_terms_per_time_step"] == terms
    assert abs(r["peak"] - 152 * 128 * 2000e6 / 1e12) < 1e-9
    assert abs(r["achieved"] - terms * 12 * 100 / 1.0 / 1e12) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["hbm"]["bytes_per_time_step"] == bench.algorithmic_bytes_per_step(
        p, p.nshots, bench.receiver_row_numbers(p), (8, 8))
    # the other modes keep the HBM roof
    assert bench.roofline_of(p, "tf32x3", t, 100, {"hbm_gbs": 7000.0}, "measured", None)["bound"] == "hbm"


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    """``bench.py --impl reference`` (the FP64 oracle on a bounded sample of
    the config-2 stepping) prints one JSON line with the contract's keys."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--cpu-sample-steps", "20"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("cfg2")
