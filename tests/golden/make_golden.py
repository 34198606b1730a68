"""Writes tests/golden/energies.json from the oracle only (no library code).

  hubbard8_dmrg_d64: the oracle's two-site DMRG (Secs. 2.3-2.4, 3.3, 4.2) on the open
      Hubbard chain L=8, N=8, S=0, t=1, U=4, C1, D=64, 6 macro-iterations, started
      from the right-normalised initial MPS of Sec. 4.3 filled by splitmix64 seed
      2415001; the minimum micro-iteration energy (Sec. 4.3) and the last one.
  hubbard8_fci: FCI (4900 determinants) of the same Hamiltonian.
  random12_fci: FCI of the L=12, N=12, S=0, Ag random-integral Hamiltonian (seed
      2415012), the reference the D=500 DMRG energy is bounded by.
Run: python tests/golden/make_golden.py [--skip-random12]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import dmrg, mps as M  # noqa: E402
from oracle.fci import FCISpace, fci_ground_state  # noqa: E402
from workloads import make_problem, uniform_pm1  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "energies.json")


def hubbard8():
    cfg, h, V = make_problem("hubbard8")
    L, N = cfg["L"], cfg["N"]
    irr = cfg["group_irreps"]
    prob = dmrg.Problem(h, V, irr, N, 0, 0)
    m = M.right_canonicalize(M.random_mps(irr, N, 0, 0, 64, uniform_pm1(2415001, 10 ** 6)))
    emin, es = dmrg.sweep(prob, m, 64, 6)
    E, vecs, space = fci_ground_state(h, V, N, 0, irr, 0)
    return {"hubbard8_dmrg_d64": {"e_min": emin, "e_last": es[-1], "seed": 2415001, "D": 64,
                                  "macro_iterations": 6},
            "hubbard8_fci": {"e": float(E[0]), "s2": float(space.s2(vecs[0]))}}


def random12():
    cfg, h, V = make_problem("random12")
    L, N = cfg["L"], cfg["N"]
    irr = cfg["group_irreps"]
    E, vecs, space = fci_ground_state(h, V, N, 0, irr, 0, dense_max=0, tol=1e-12)
    C = vecs[0]
    return {"random12_fci": {"e": float(E[0]), "n_det": int(space.mask.sum()),
                             "s2": float(np.vdot(C, space.s2_apply(C)) / np.vdot(C, C))}}


if __name__ == "__main__":
    res = json.load(open(OUT)) if os.path.exists(OUT) else {}
    t = time.time()
    res.update(hubbard8())
    print("hubbard8 done", time.time() - t, flush=True)
    if "--skip-random12" not in sys.argv:
        res.update(random12())
        print("random12 done", time.time() - t, flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(json.dumps(res, indent=1))
