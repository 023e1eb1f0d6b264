"""Write the regression fixtures in this folder from the oracle alone.

The values are oracle outputs, not values printed in the paper (the paper
gives no worked numerical example of the residual): they pin the seeded
generator and the oracle against unintended change.  The oracle itself is
pinned by closed forms and invariants in tests/test_oracle_pins.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import closed_shell as cs, solver as osolver, thc  # noqa: E402
from synth import make_system, random_amplitudes  # noqa: E402

CASES = [(3, 7, 10, 14, 9, 5), (5, 20, 60, 120, 60, 0)]


def fingerprint(s):
    """Frobenius norms and first entries of the generated inputs."""
    arrs = (s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z)
    return [[float(np.linalg.norm(a)), float(a.ravel()[0])] for a in arrs]


def case_values(o, v, P, G, K, seed):
    s = make_system(o, v, P, G, K, seed)
    Zc, t1 = random_amplitudes(P, o, v, seed + 1000, t2_scale=0.05, t1_scale=0.05)
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    r1, sig = osolver.projected_residual(H, s.Y, Zc, t1)
    E = cs.energy(H, t1, thc.amplitudes(s.Y, Zc, o))
    return {"case": [o, v, P, G, K, seed], "inputs": fingerprint(s),
            "energy": E, "sigma_fro": float(np.linalg.norm(sig)),
            "sigma1_fro": float(np.linalg.norm(r1)), "sigma_00": float(sig[0, 0]),
            "sigma1_00": float(r1[0, 0]), "mp2": osolver.mp2_energy(H, s.eps_o, s.eps_v)}


def main():
    out = {"source": "oracle/ (FP64 numpy), written by tests/golden/make_golden.py",
           "cases": [case_values(*c) for c in CASES]}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
