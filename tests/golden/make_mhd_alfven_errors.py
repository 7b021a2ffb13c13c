"""Writes mhd_alfven_errors.json: the oracle's errors against the exact
Alfven wave (3D ideal MHD, weak form + Powell term + LLF, N = 3, CFL 0.5
step from the initial state, held fixed as T / steps) after LSRK steps to
T = 0.1 on 16^3 and 32^3 elements. Calls only the oracle and the input
generators; run from the repository root:

    python tests/golden/make_mhd_alfven_errors.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as orc  # noqa: E402
from paper_2108_06476_gb300 import workloads as W  # noqa: E402

G, N, T = 5.0 / 3.0, 3, 0.1


def run(ne):
    n = (ne, ne, ne)
    xi, _ = orc.lgl(N)
    u = W.alfven_wave(N, n, xi, 0.0, gamma=G)
    dt0 = orc.mhd_max_dt(N, n, W.box(3), u, 0.5, G)
    steps = int(math.ceil(T / dt0))
    for _ in range(steps):
        u = orc.mhd_lsrk_step(N, n, W.box(3), u, T / steps, G, True)
    e = u - W.alfven_wave(N, n, xi, T, gamma=G)
    return {"steps": steps, "dt0": dt0, "max_err": float(np.abs(e).max()),
            "rms_err": float(np.sqrt(np.mean(e * e)))}


if __name__ == "__main__":
    out = {"source": "oracle (dgsem_mhd.c) via make_mhd_alfven_errors.py",
           "problem": "Alfven wave, gamma 5/3, N = 3, T = 0.1, CFL 0.5, Powell term, LLF"}
    for ne in (16, 32):
        out[str(ne)] = run(ne)
        print(ne, out[str(ne)], flush=True)
    with open(os.path.join(HERE, "mhd_alfven_errors.json"), "w") as fh:
        json.dump(out, fh, indent=1)
