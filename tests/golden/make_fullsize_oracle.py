"""Write the FP64 oracle's results for the full-size workloads to tests/golden/.

Runs the oracle (and only the oracle) on the seeded inputs of gen/ and stores,
per workload, in fullsize_<key>.npz:

  E_x      the exchange energy over every listed pair (Eq. 4)
  M        Phi^T W (Section 2.2); all rows for the water boxes, the rows
           M_rows for the 512-orbital localised box
  M_rows   which rows of M are stored
  Kpsi     K t for the first n_kpsi trial vectors, K = -xi xi^T built by the
           oracle's own Cholesky route (Eq. 5), rounded to complex64 (the
           comparison tolerance is 1e-6 of the maximum; complex64 rounding
           is 6e-8 of each element)
  Q        t_m^T K t_n over n_q trial vectors (the operator as a quadratic
           form, FP64)
  trials_seed, n_kpsi, n_q: how the trials are drawn (gen.random_trials)
  meta     JSON: workload name, this script's SHA-256, oracle wall seconds

Usage:  python tests/golden/make_fullsize_oracle.py water32 [water64 localized] [--threads N]
The water32 workload takes about 15 minutes on 8 cores, water64 and
localized one to two hours each.
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(_HERE)))

import gen  # noqa: E402
import oracle  # noqa: E402

TRIALS_SEED = 909
WORKLOADS = {
    # key: (config function, rows of M stored (None = all), trials with K psi stored, trials of Q)
    "water32": (gen.config_water32, None, 2, 16),
    "water64": (lambda: gen.config_water64(n_trial_sets=0), None, 1, 16),
    "localized": (gen.config_localized, list(range(0, 512, 32)), 1, 16),
}


def script_sha256():
    with open(os.path.abspath(__file__), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def path_for(key):
    return os.path.join(_HERE, f"fullsize_{key}.npz")


def make(key, nthreads):
    fn, rows, n_kpsi, n_q = WORKLOADS[key]
    cfg = fn()
    t0 = time.time()
    ref = oracle.ace_build(cfg["psi"], cfg["cell"], cfg["grid"], cfg["ecut"], cfg["alpha"], pairs=cfg.get("pairs"),
                           nthreads=nthreads)
    t_build = time.time() - t0
    trials = gen.random_trials(cfg["cell"], cfg["ecut"], max(n_kpsi, n_q), seed=TRIALS_SEED)
    K = oracle.ace_apply(ref["xi"], trials, ref["miller"])
    Q = gen.gamma_overlap(trials[:n_q], K[:n_q])
    M = ref["M"] if rows is None else ref["M"][rows]
    meta = dict(workload=cfg["name"], script=os.path.basename(__file__), script_sha256=script_sha256(),
                oracle_build_s=round(t_build, 1), threads=nthreads)
    np.savez(path_for(key), E_x=np.float64(ref["E_x"]), M=M,
             M_rows=np.arange(len(cfg["psi"])) if rows is None else np.array(rows),
             Kpsi=K[:n_kpsi].astype(np.complex64), Q=Q, trials_seed=TRIALS_SEED, n_kpsi=n_kpsi, n_q=n_q,
             meta=json.dumps(meta))
    print(f"{key}: E_x = {ref['E_x']:.12f} in {t_build:.0f} s -> {path_for(key)}", flush=True)


def load(key):
    """The stored results of one workload as a dict (meta decoded)."""
    with np.load(path_for(key)) as z:
        d = {k: z[k] for k in z.files}
    d["meta"] = json.loads(str(d["meta"]))
    d["E_x"] = float(d["E_x"])
    return d


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("keys", nargs="+", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    for k in a.keys:
        make(k, a.threads)
