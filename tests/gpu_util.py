"""Helpers shared by the GPU tests (no test functions here)."""
import numpy as np

from synth import make_system, random_amplitudes
from oracle import closed_shell as cs, solver as osolver, thc


def oracle_case(o, v, P, G, K, seed, t1_scale=0.05, t2_scale=0.05, consistent=False):
    s = make_system(o, v, P, G, K, seed, consistent=consistent)
    Zc, t1 = random_amplitudes(P, o, v, seed + 1000, t2_scale=t2_scale, t1_scale=t1_scale)
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    r1, sig = osolver.projected_residual(H, s.Y, Zc, t1)
    E = cs.energy(H, t1, thc.amplitudes(s.Y, Zc, o))
    return s, Zc, t1, sig, r1, E


def context(s, **kw):
    import paper_2111_11473_gb300 as pkg
    return pkg.Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z, **kw)
