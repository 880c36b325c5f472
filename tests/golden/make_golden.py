"""Write oracle results for the CTMRG workloads to tests/golden/ctmrg_w<k>.json.

Calls only the oracle (dense FP64 CPU CTMRG) on the seeded inputs. Usage:
    python tests/golden/make_golden.py 1 2 3
Stored per checkpoint (number of moves): the Heisenberg bond energy, the
normalised two-site RDM, the normalised corner spectrum, the symmetry error
of Eq. (4), and per move the relative gap at the truncation cut.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ctmrg, doublelayer as dl, observables as ob  # noqa: E402
from paper_2410_11596_gb300 import inputs  # noqa: E402

CHECKPOINTS = (1, 2, 3, 5, 10, 20, 30, 40, 50)


def snapshot(C, T, A, D):
    # D >= 7: the two-site network summed over slices of its bottom bond, and no
    # S_err (the one-site environment's chi^2 D^6 intermediate is tens of GB)
    big = D >= 7
    rho = ob.two_site_rdm(C, T, A, chunk=8 if big else None)
    rho = rho / np.trace(rho)
    out = {
        "energy": ob.bond_energy(rho, inputs.heisenberg_bond()),
        "rho_re": np.real(rho).tolist(),
        "rho_im": np.imag(rho).tolist(),
        "corner_spectrum": ob.corner_spectrum(C).tolist(),
    }
    out["s_err"] = None if big else ob.symmetry_error(ob.one_site_environment(C, T), D)
    return out


def compute(k, verbose=False):
    """The stored record of workload k, computed by the oracle."""
    w = inputs.WORKLOADS[k]
    A = inputs.workload_tensor(k)
    a = dl.double_layer(A)
    C, T = ctmrg.init_environment(a)
    C, T = C / np.abs(C).max(), T / np.abs(T).max()
    res = {"workload": k, **w, "seed": w.get("seed", inputs.SEED_BASE + k), "checkpoints": {}, "gaps": [], "lam_cut": [],
           "n": []}
    t0 = time.time()
    for m in range(1, w["moves"] + 1):
        C, T, info = ctmrg.move(C, T, a, w["chi"])
        res["gaps"].append(float(info.gap) if np.isfinite(info.gap) else None)
        res["lam_cut"].append(info.lam_cut)
        res["n"].append(info.n)
        if m in CHECKPOINTS or m == w["moves"]:
            res["checkpoints"][str(m)] = snapshot(C, T, A, w["D"])
            if verbose:
                print(f"w{k} move {m} E={res['checkpoints'][str(m)]['energy']:.15f} t={time.time()-t0:.1f}s",
                      flush=True)
    res["oracle_seconds"] = time.time() - t0
    return res


def main(ks):
    for k in ks:
        res = compute(k, verbose=True)
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"ctmrg_w{k}.json")
        with open(path, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main([int(x) for x in sys.argv[1:]] or [1, 2])
