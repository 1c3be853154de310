"""Mechanical mutation sweeps of the oracle (test infrastructure; not collected
by pytest).  Each sweep changes one thing on every code line of
oracle/mpm_oracle.c (or oracle/mlp.py) in a private copy, runs the oracle's pin suite on the copy
and lists the copies that still pass:

    python tests/oracle_sweep.py ops      # swap the first binary +, -, * of a line
    python tests/oracle_sweep.py consts   # move the first literal 0.5 ... 9.0 of a line
    python tests/oracle_sweep.py index    # transpose the first index pair of a line
    python tests/oracle_sweep.py mlp      # swap +, -, *, / or drop a .T in oracle/mlp.py

Survivors are either equivalent (they cannot change any result) or a missing
pin; tests/test_oracle_mutations.py keeps a representative copy of every
mistake a sweep showed the pins missing.
"""
from __future__ import annotations

import os
import re
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_mutations as harness  # noqa: E402

OPS = ((" + ", " - "), (" - ", " + "), (" * ", " / "))
CONSTS = (("0.5", "0.25"), ("2.0", "1.0"), ("3.0", "2.0"), ("1.0", "2.0"), ("1.5", "1.25"), ("0.75", "0.7"),
          ("6.0", "5.0"), ("9.0", "8.0"))
INDEX = (("[a * d + b]", "[b * d + a]"), ("[b * d + a]", "[a * d + b]"), ("[i * 3 + j]", "[j * 3 + i]"),
         ("[j * 3 + k]", "[k * 3 + j]"), ("[i * 3 + k]", "[k * 3 + i]"), ("[k * 3 + l]", "[l * 3 + k]"),
         ("[a * 3 + b]", "[b * 3 + a]"), ("[b * 3 + a]", "[a * 3 + b]"), ("[a * d + c]", "[c * d + a]"),
         ("[b * d + c]", "[c * d + b]"), ("[i * d + a]", "[a * d + i]"), ("[i * d + k]", "[k * d + i]"),
         ("[k * d + j]", "[j * d + k]"))


MLP_OPS = ((" + ", " - "), (" - ", " + "), (" * ", " / "), (" / ", " * "), (".T", ""))


def mutants(lines, kind):
    out = []
    if kind == "mlp":
        for i, line in enumerate(lines):
            s = line.strip()
            if not s or s.startswith(("#", '"""', "def ", "import", "from")):
                continue
            for old, new in MLP_OPS:
                k = line.find(old)
                if k >= 0:
                    out.append((i, old, new, k))
        return out
    for i, line in enumerate(lines):
        s = line.strip()
        if not s or s.startswith(("/*", "*", "//", "#")):
            continue
        code = line.split("/*")[0]
        if kind == "ops":
            for old, new in OPS:
                k = code.find(old)
                if k >= 0:
                    out.append((i, old, new, k))
        elif kind == "consts":
            for old, new in CONSTS:
                m = re.search(r"(?<![0-9.e])" + re.escape(old) + r"(?![0-9])", code)
                if m:
                    out.append((i, old, new, m.start()))
        else:
            for old, new in INDEX:
                k = code.find(old)
                if k >= 0:
                    out.append((i, old, new, k))
    return out


def run(kind: str, workers: int = 8):
    fname = "mlp.py" if kind == "mlp" else "mpm_oracle.c"
    pins = harness.MLP_PINS if kind == "mlp" else harness.C_PINS
    src = open(os.path.join(harness.ROOT, "oracle", fname)).read()
    lines = src.split("\n")
    muts = mutants(lines, kind)

    def one(m):
        i, old, new, k = m
        mutated = list(lines)
        mutated[i] = mutated[i][:k] + new + mutated[i][k + len(old):]
        with tempfile.TemporaryDirectory(prefix="oracle_sweep_") as tmp:
            base = harness._tree(os.path.join(tmp, "b"))
            with open(os.path.join(base, "oracle", fname), "w") as fh:
                fh.write("\n".join(mutated))
            try:
                rc = harness._run(base, pins).returncode
            except RuntimeError:
                rc = "no build"
        return i, old, rc

    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(one, muts))
    survivors = [(i + 1, old, lines[i].strip()) for i, old, rc in res if rc == 0]
    crashed = [(i + 1, old, rc) for i, old, rc in res if rc not in (0, 1)]
    print(f"{kind}: {len(muts)} copies, {len(muts) - len(survivors) - len(crashed)} caught, "
          f"{len(survivors)} survived, {len(crashed)} crashed")
    for s in survivors:
        print("  survived: line %d %r: %s" % s)
    return survivors


if __name__ == "__main__":
    run(sys.argv[1] if len(sys.argv) > 1 else "ops")
