"""Write oracle_reference.json: FP64 oracle results on the benchmark workloads.

Calls only the input generator and oracle/ (plus scipy's eigen-solver for the
exact minimum 2 * sum of the n lowest generalised eigenvalues).  The stored
iteration counts let the CPU-baseline arm time a bounded sample of oracle CG
steps and scale it to a full solve; the stored energies let the benchmark
report its accuracy without re-running the oracle.

    python tests/golden/make_oracle_reference.py [c1] [c2]
"""
import json
import os
import sys
import time

import numpy as np
import scipy.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import omm as O  # noqa: E402

WORKLOADS = {
    "c1": dict(dims=(4, 4, 4), seed=0, tol=1e-10),
    "c2": dict(dims=(8, 8, 8), seed=0, tol=1e-10),
}


def run(name):
    w = WORKLOADS[name]
    sysm = synth.make_system(*w["dims"], seed=w["seed"])
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    lam = sla.eigh(H, S, eigvals_only=True, subset_by_index=[0, sysm.n])
    t0 = time.time()
    res = O.omm_cg(H, S, W0, tol=w["tol"])
    t = time.time() - t0
    e_exact = 2.0 * float(np.sum(lam[:sysm.n]))
    # density matrix rho = 2 W (2I - S_W) W^T (Eq. 5) of the oracle's solve, and the
    # exact one, 2 V V^T over the S-orthonormal lowest-n eigenvectors, on sampled
    # entries (the full m x m matrix is too large to store)
    rng = np.random.default_rng(7)
    m, n = sysm.m, sysm.n
    idx = np.concatenate([rng.integers(0, m, (1500, 2)), np.repeat(rng.integers(0, m, (100, 1)), 2, axis=1)])
    W = np.asarray(res.W)
    K = 2.0 * np.eye(n) - W.T @ (S @ W)
    rho_oracle = 2.0 * np.einsum("ka,ab,kb->k", W[idx[:, 0]], K, W[idx[:, 1]])
    _, V = sla.eigh(H, S, subset_by_index=[0, n - 1])
    rho_exact = 2.0 * np.einsum("ka,ka->k", V[idx[:, 0]], V[idx[:, 1]])
    return {
        "dims": list(w["dims"]), "seed": w["seed"], "m": sysm.m, "n": sysm.n, "tol": w["tol"],
        "eta_gershgorin": res.eta, "oracle_iters": res.iters, "oracle_E": res.E,
        "exact_E": e_exact, "lambda_n": float(lam[sysm.n - 1]), "lambda_n_plus_1": float(lam[sysm.n]),
        "oracle_rel_err": abs(res.E - e_exact) / abs(e_exact), "oracle_seconds_here": t,
        "rho_samples": {"idx": idx.tolist(), "oracle": rho_oracle.tolist(), "exact": rho_exact.tolist(),
                        "max_abs_oracle_vs_exact": float(np.abs(rho_oracle - rho_exact).max())},
    }


if __name__ == "__main__":
    out_path = os.path.join(HERE, "oracle_reference.json")
    data = json.load(open(out_path)) if os.path.exists(out_path) else {}
    for name in (sys.argv[1:] or list(WORKLOADS)):
        data[name] = run(name)
        print(name, data[name])
        json.dump(data, open(out_path, "w"), indent=1, sort_keys=True)
