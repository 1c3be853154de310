"""The byte accounting behind bench.py's roofline figures, checked on the CPU:
the active-node count against a brute-force set of stencil nodes, the
algorithmic bytes per particle against the state components each kernel must
move, the DRAM traffic file's format, and the parsing of the clock record
taken during the timed region (median SM clock, maximum clock, throttle
reasons that were active)."""
import os
import subprocess
import tempfile

import numpy as np

import bench


def test_active_nodes_match_brute_force():
    rng = np.random.default_rng(0)
    n_cells = (10, 7, 5)
    dx = 0.1
    x = rng.uniform(0, 1, (300, 3)) * np.array(n_cells) * dx
    x[:5] = 0.0                                   # particles on the walls and corners
    x[5:10] = np.array(n_cells) * dx
    nodes = set()
    for p in x:
        b = np.floor(p / dx - 0.5).astype(int)
        for off in np.ndindex(3, 3, 3):
            nodes.add(tuple(b + np.array(off)))
    assert bench.count_active_nodes(x, dx, n_cells) == len(nodes)


def test_algorithmic_bytes_per_particle():
    # 3D Drucker-Prager FP32: P2G reads x v C rho sigma (22 words); G2P reads x F rho
    # sigma eps (20) and writes the whole 32-word state
    assert bench.algorithmic_bytes_per_particle("p2g", 3, 1, 4) == 22 * 4
    assert bench.algorithmic_bytes_per_particle("g2p", 3, 1, 4) == (20 + 32) * 4
    # 2D fluid FP64: P2G x v C rho (9 words); G2P x F rho (7) read, 13 written
    assert bench.algorithmic_bytes_per_particle("p2g", 2, 0, 8) == 9 * 8
    assert bench.algorithmic_bytes_per_particle("g2p", 2, 0, 8) == (7 + 13) * 8


def test_traffic_file_lists_the_roofline_kernels():
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.txt")
    assert os.path.exists(path)
    for k in ("p2g", "g2p"):
        v = bench.read_traffic(k)
        assert v is None or v > 0


def test_clock_record_parsing():
    rows = ["0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1995, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, [N/A], 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2040, 2070, 1200.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
            "garbage line"]
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    cs = object.__new__(bench.ClockSampler)
    cs.path, cs.gpu = path, 0
    cs.fh = open(os.devnull, "w")
    cs.proc = subprocess.Popen(["sleep", "30"])
    out = cs.stop()
    assert out == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 4}
    assert not os.path.exists(path)


def test_clock_records_that_reject_a_number():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 50}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"], sm_mhz=1800.0))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))          # stuck low with no reason: a clock lock
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1900.0))
