"""Readers for the hand-written fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def peak_cases():
    """Yield dicts(name, T, max_peaks, found, acc, expect[list of (t, b, v)])."""
    with open(os.path.join(GOLDEN, "peaks_cases.txt")) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    i = 0
    while i < len(lines):
        ln = lines[i].strip()
        i += 1
        if not ln:
            continue
        assert ln.startswith("case "), ln
        parts = ln.split()
        kv = dict(p.split("=") for p in parts[2:])
        rows = []
        while not lines[i].strip().startswith("expect"):
            rows.append([int(x) for x in lines[i].split()])
            i += 1
        exp = [tuple(int(x) for x in tok.split(",")) for tok in lines[i].split()[1:]]
        i += 1
        assert lines[i].strip() == "end"
        i += 1
        yield dict(name=parts[1], T=int(kv["T"]), max_peaks=int(kv["max_peaks"]),
                   found=int(kv["found"]), acc=np.array(rows, np.int32), expect=exp)


def geometry_facts():
    out = {}
    with open(os.path.join(GOLDEN, "geometry.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            k, v = ln.split()[:2]
            out[k] = float(v)
    return out
