"""A plain C program using only include/hough.h, libhough.so and the CUDA
runtime finds the same peaks and assignments as the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import build, synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_c_client_matches_oracle(tmp_path):
    lib = build.build()
    cuda = os.path.dirname(os.path.dirname(build.nvcc()))
    exe = tmp_path / "find_windows"
    subprocess.run(["gcc", "-std=c11", "-O2", "-I", os.path.join(build.ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(HERE, "c", "find_windows.c"),
                    "-o", str(exe), "-L", os.path.dirname(lib), "-lhough",
                    "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-Wl,-rpath," + os.path.dirname(lib) + ":" + os.path.join(cuda, "lib64")],
                   check=True)
    w = synth.workload("plain", n_windows=40, seed=17)
    data = tmp_path / "windows.bin"
    with open(data, "wb") as fh:
        np.array([w.n_windows, 512, 512], np.int64).tofile(fh)
        w.offsets.astype(np.int64).tofile(fh)
        w.vane.astype(np.int32).tofile(fh)
        w.strip.astype(np.int32).tofile(fh)
    out = subprocess.run([str(exe), str(data)], check=True, capture_output=True, text=True).stdout
    lines = out.splitlines()
    phi, z = oracle.encode(synth.GEOMETRY, w.vane, w.strip)
    ref = oracle.find_batch(synth.GEOMETRY, 512, 512, phi, z, w.offsets)
    i = 0
    for k in range(w.n_windows):
        wk, npk, nfd, st = (int(x) for x in lines[i].split())
        i += 1
        assert (wk, npk, nfd, st) == (k, ref["n_peaks"][k], ref["n_found"][k], ref["status"][k])
        for j in range(npk):
            got = tuple(int(x) for x in lines[i].split())
            i += 1
            e = ref["peaks"][k][j]
            assert got == (e["theta"], e["rho"], e["votes"], e["n_hits"], e["hit_begin"])
        ht = [int(x) for x in lines[i].split()]
        i += 1
        assert ht == list(ref["hit_track"][w.window(k)])
