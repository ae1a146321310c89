"""The stored full-size oracle values (tests/golden/fullsize_*.npz): each was
written by the committed make_fullsize_oracle.py (its SHA-256 in the file's
metadata), for the workload the key names, with the shapes the GPU tests
compare against, and with invariants the oracle's M and Q must satisfy
(M = Phi^T W is symmetric with a negative diagonal, and its trace is E_x when
every pair is listed; Q = t^T K t is a symmetric negative semidefinite form
since K = -xi xi^T)."""
import hashlib
import os
import sys

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, HERE)
import make_fullsize_oracle as mfo  # noqa: E402

SIZES = {"water32": 128, "water64": 256, "localized": 512}


@pytest.mark.parametrize("key", sorted(SIZES))
def test_fullsize_golden_file(key):
    d = mfo.load(key)
    with open(os.path.join(HERE, "make_fullsize_oracle.py"), "rb") as f:
        assert d["meta"]["script_sha256"] == hashlib.sha256(f.read()).hexdigest()
    fn, rows, n_kpsi, n_q = mfo.WORKLOADS[key]
    n = SIZES[key]
    assert d["meta"]["workload"].startswith(key)
    assert list(d["M_rows"]) == (list(range(n)) if rows is None else rows)
    assert d["M"].shape == (len(d["M_rows"]), n)
    assert d["Kpsi"].shape[0] == n_kpsi == int(d["n_kpsi"]) and d["Q"].shape == (n_q, n_q)
    assert int(d["trials_seed"]) == mfo.TRIALS_SEED
    assert np.isfinite(d["E_x"]) and d["E_x"] < 0
    # M on the stored rows: negative diagonal; symmetric where both rows are stored
    diag = d["M"][np.arange(len(d["M_rows"])), d["M_rows"]]
    assert (diag < 0).all()
    if rows is None:
        assert np.abs(d["M"] - d["M"].T).max() <= 1e-10 * np.abs(d["M"]).max()
        # with every pair listed, E_x = -alpha sum_{i<=j} (2 - d_ij) e_ij (Eq. 4) is
        # -alpha sum_{i,j} e_ij, and M_ii = <phi_i|W_i> = -alpha sum_j <phi_i|v_ij phi_j>
        # = -alpha sum_j e_ij (Eq. 2): E_x = tr M, two separate oracle routes
        assert abs(d["E_x"] - np.trace(d["M"])) <= 1e-10 * abs(d["E_x"])
    Q = d["Q"]
    assert np.abs(Q - Q.T).max() <= 1e-9 * np.abs(Q).max()
    assert np.linalg.eigvalsh(0.5 * (Q + Q.T)).max() <= 1e-9 * np.abs(Q).max()
