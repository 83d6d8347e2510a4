"""Write the full-size expected histograms used by the GPU parity tests.

Every value here comes from the FP64 oracle (oracle/cf_oracle.c, z-window mode, which the pins
show to be bit-identical to brute force) run on the seeded synthetic workloads of gen/.  The
file also records a fingerprint of the generated arrays, so a test on another machine can tell
whether its generator produced the same inputs.

    python tests/golden/make_golden.py [name ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402

BATCH_SAMPLE = [0, 1, 2, 3]          # catalogues of the 256-catalogue batch given golden values


def fingerprint(*cats) -> str:
    h = hashlib.sha256()
    for c in cats:
        if c is None:
            continue
        for a in (c.x, c.y, c.z, c.w):
            if a is not None:
                h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def batch_names():
    sizes = gen.batch_sizes()
    order = np.argsort(sizes)
    pick = sorted(set([int(order[0]), int(order[-1])] + BATCH_SAMPLE))
    return [f"batch_{i}" for i in pick]


def workload(name):
    if name.startswith("batch_"):
        i = int(name.split("_")[1])
        n = gen.batch_sizes()[i]
        cat = gen.batch_catalogue(i, n)
        return gen.Workload(name, "rppi", True, True, 250.0, gen.log_edges(0.1, 20.0, 14), cat,
                            pimax=40.0, npibins=40)
    return gen.workload(name)


def make(name: str) -> dict:
    wl = workload(name)
    t0 = time.time()
    out = oracle.count(wl.kind, wl.edges, wl.d1, None if wl.autocorr else wl.d2, autocorr=wl.autocorr,
                       periodic=wl.periodic, box=wl.box, pimax=wl.pimax, npibins=wl.npibins, weighted=wl.weighted,
                       ravg=wl.ravg, mode="zwin")
    rec = {
        "name": name,
        "gen_version": gen.GEN_VERSION,
        "fingerprint": fingerprint(wl.d1, wl.d2),
        "oracle_mode": "zwin",
        "oracle_seconds": round(time.time() - t0, 1),
        "npairs": [int(v) for v in np.asarray(out["npairs"]).ravel()],
        "wsum": [float(v) for v in np.asarray(out["wsum"]).ravel()],
    }
    if "ravg" in out:
        rec["ravg"] = [float(v) for v in np.asarray(out["ravg"]).ravel()]
    return rec


def main(names):
    if not names:
        names = ["clustered_r_1m", "sphere_theta_1m", "clustered_rppi_2m", "clustered_wp_2m"] + batch_names() + \
                ["clustered_rppi_dr", "mock_dr_rppi", "clustered_rppi_2m_wr"]
    for name in names:
        path = os.path.join(HERE, f"full_{name}.json")
        rec = make(name)
        with open(path, "w") as f:
            json.dump(rec, f)
        print(name, rec["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
