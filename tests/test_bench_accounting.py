"""The byte accounting behind bench.py's roofline figures, checked on the CPU:
the active-node count against a brute-force set of stencil nodes, the
algorithmic bytes per particle against the state components each kernel must
move, and the DRAM traffic file's format."""
import os

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
