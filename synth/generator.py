"""Synthetic THC-RR-CCSD systems shaped like the paper's workloads.

The paper's molecules, basis sets and integrals are not available, so every
input is drawn from a seeded generator:

* occupied orbital energies  eps_o ~ U[-1.5, -0.3] Eh, sorted ascending;
* virtual orbital energies   eps_v ~ U[ 0.1,  3.0] Eh, sorted ascending;
* ERI grid collocation       x ~ N(0,1)/sqrt(G), shape (n, G);
* grid metric factor          A = |N(0,1)| * sqrt(gamma / (K * 2/pi)), shape (G, K);
* amplitude collocation      Y ~ N(0,1)/sqrt(P), shape (n, P);
  drawn in that order from ``numpy.random.default_rng(seed)``.

The generator's text leaves the scale and sign of A open.  A non-negative A
makes the grid kernel z elementwise positive, like the Coulomb kernel 1/r12
it stands for, and the scale puts Coulomb-type integrals (pp|qq) near
``gamma`` (default 0.3 Eh) while ovov integrals stay of order gamma / G, so
the amplitude equations are well conditioned at every size.

Derived inputs (input construction, not the method):

* ERI-THC core  z = A A^T + 1e-3 I   (G x G, the THC form of Eq. 17);
* R = first K columns of a diagonally pivoted Cholesky factor of z (G x K);
* Cholesky vectors  L[K, p, q] = sum_I x[p, I] x[q, I] R[I, K]   (Eq. 24).

With ``consistent=True`` the Cholesky rank is the full grid size (K = G) and
the Cholesky and THC ovov integrals agree exactly; the invariant tests use it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    """One synthetic closed-shell system (all arrays float64, C order)."""
    o: int
    v: int
    P: int
    G: int
    K: int
    seed: int
    eps_o: np.ndarray   # (o,)
    eps_v: np.ndarray   # (v,)
    Y: np.ndarray       # (n, P) occupied rows first
    x: np.ndarray       # (n, G)
    z: np.ndarray       # (G, G) symmetric
    L: np.ndarray       # (K, n, n) symmetric in the last two indices

    @property
    def n(self) -> int:
        return self.o + self.v


def _pivoted_cholesky(V: np.ndarray, rank: int) -> np.ndarray:
    """Diagonally pivoted (outer-product) Cholesky: V ~= R R^T, R is G x rank.

    Columns come in pivot order (largest remaining diagonal first).
    """
    G = V.shape[0]
    R = np.zeros((G, rank))
    d = np.diag(V).astype(np.float64).copy()
    for k in range(rank):
        p = int(np.argmax(d))
        piv = d[p]
        if piv <= 0.0:
            break
        col = V[:, p] - R[:, :k] @ R[p, :k]
        col /= np.sqrt(piv)
        R[:, k] = col
        d -= col * col
        d[p] = 0.0
    return R


def make_system(o: int, v: int, P: int, G: int, K: int, seed: int,
                consistent: bool = False, gamma: float = 0.3) -> System:
    """Draw one synthetic system.  ``consistent`` forces K = G."""
    if consistent:
        K = G
    rng = np.random.default_rng(seed)
    eps_o = np.sort(rng.uniform(-1.5, -0.3, o))
    eps_v = np.sort(rng.uniform(0.1, 3.0, v))
    n = o + v
    x = rng.standard_normal((n, G)) / np.sqrt(G)
    A = np.abs(rng.standard_normal((G, K))) * np.sqrt(gamma / (K * 2.0 / np.pi))
    Y = rng.standard_normal((n, P)) / np.sqrt(P)
    z = A @ A.T + 1e-3 * np.eye(G)
    z = 0.5 * (z + z.T)
    R = _pivoted_cholesky(z, K)
    # L[K, p, q] = sum_I x[p, I] x[q, I] R[I, K], built one Cholesky vector
    # at a time to bound the temporary.
    L = np.empty((K, n, n))
    for k in range(K):
        L[k] = (x * R[:, k]) @ x.T
    L = 0.5 * (L + L.transpose(0, 2, 1))
    return System(o, v, P, G, K, seed, eps_o, eps_v,
                  np.ascontiguousarray(Y), np.ascontiguousarray(x),
                  np.ascontiguousarray(z), np.ascontiguousarray(L))


@dataclass
class DeviceSystem:
    """A system whose Cholesky vectors are formed on a torch device, a slab
    at a time (the 2500-basis shape has 375 GB of them in float64).  Same
    draws as ``make_system``; z and the pivoted Cholesky factor R are formed
    on the device in float64, the vectors in float32 (the precision the
    mixed-precision engine stores them in)."""
    o: int
    v: int
    P: int
    G: int
    K: int
    seed: int
    eps_o: np.ndarray   # (o,)
    eps_v: np.ndarray   # (v,)
    Y: np.ndarray       # (n, P)
    x: np.ndarray       # (n, G)
    z: np.ndarray       # (G, G)
    Rt: object          # torch (K, G) float64 on the device: column k of R is row k
    L = None

    @property
    def n(self) -> int:
        return self.o + self.v

    def cholesky_slabs(self, nk: int = 32, k_lo: int = 0, k_hi=None):
        """Yield (k0, L[k0:k0+nk]) as float64 (nk, n, n) device tensors with
        L[k, p, q] = sum_I x[p, I] x[q, I] R[I, k] formed in float32 and
        symmetrised, for the vectors k_lo .. k_hi - 1 (default: all)."""
        import torch
        dev = self.Rt.device
        xf = torch.from_numpy(self.x).to(dev, torch.float32)
        n = self.n
        k_hi = self.K if k_hi is None else k_hi
        for k0 in range(k_lo, k_hi, nk):
            kk = min(nk, k_hi - k0)
            # M[k, q, I] = R[I, k] x[q, I];  L[k] = M[k] x^T
            M = self.Rt[k0:k0 + kk].to(torch.float32)[:, None, :] * xf[None, :, :]
            Lk = (M.reshape(kk * n, self.G) @ xf.T).reshape(kk, n, n)
            del M
            Lk = 0.5 * (Lk + Lk.transpose(1, 2))
            yield k0, Lk.to(torch.float64)
            del Lk


def _pivoted_cholesky_torch(V, rank: int):
    """``_pivoted_cholesky`` on a torch tensor, without host synchronisation:
    returns R^T (rank x G)."""
    import torch
    G = V.shape[0]
    Rt = torch.zeros((rank, G), dtype=V.dtype, device=V.device)
    d = V.diagonal().clone()
    for k in range(rank):
        p = torch.argmax(d).view(1)
        piv = d.index_select(0, p)
        col = V.index_select(0, p)[0] - Rt[:k].T @ Rt[:k].index_select(1, p)[:, 0]
        col = col / torch.sqrt(piv)
        Rt[k] = col
        d -= col * col
        d.index_fill_(0, p, 0.0)
    return Rt


def make_device_system(o: int, v: int, P: int, G: int, K: int, seed: int, device,
                       gamma: float = 0.3) -> DeviceSystem:
    """``make_system`` with z, R and the Cholesky vectors formed on ``device``
    (the vectors lazily, through ``DeviceSystem.cholesky_slabs``)."""
    import torch
    rng = np.random.default_rng(seed)
    eps_o = np.sort(rng.uniform(-1.5, -0.3, o))
    eps_v = np.sort(rng.uniform(0.1, 3.0, v))
    n = o + v
    x = rng.standard_normal((n, G)) / np.sqrt(G)
    A = np.abs(rng.standard_normal((G, K))) * np.sqrt(gamma / (K * 2.0 / np.pi))
    Y = rng.standard_normal((n, P)) / np.sqrt(P)
    At = torch.from_numpy(A).to(device)
    del A
    z = At @ At.T
    del At
    z.diagonal().add_(1e-3)
    z = 0.5 * (z + z.T)
    Rt = _pivoted_cholesky_torch(z, K)
    zh = z.cpu().numpy()
    del z
    return DeviceSystem(o, v, P, G, K, seed, eps_o, eps_v, np.ascontiguousarray(Y),
                        np.ascontiguousarray(x), np.ascontiguousarray(zh), Rt)


def random_amplitudes(P: int, o: int, v: int, seed: int,
                      t2_scale: float = 1e-2, t1_scale: float = 1e-2):
    """A symmetric THC core Zc (P x P) and singles t1 (o x v).

    Zc has entries of size ``t2_scale * P`` so that the doubles amplitudes it
    encodes are of size ``t2_scale`` when Y ~ N(0,1)/sqrt(P).
    """
    rng = np.random.default_rng(seed)
    Zc = rng.standard_normal((P, P)) * (t2_scale * P)
    Zc = 0.5 * (Zc + Zc.T)
    t1 = rng.standard_normal((o, v)) * t1_scale
    return np.ascontiguousarray(Zc), np.ascontiguousarray(t1)


# The workloads, named by their sizes: (o, v, P, G, K, seed).
CONFIGS = {
    "o5_v20_P60_G120_K60": (5, 20, 60, 120, 60, 0),
    "o40_v200_P400_G1200_K600": (40, 200, 400, 1200, 600, 1),
    # half the bench size in every dimension (kernel profiles of a few GB)
    "o20_v100_P200_G600_K300": (20, 100, 200, 600, 300, 1),
    "o100_v600_P1000_G3500_K1500": (100, 600, 1000, 3500, 1500, 2),
    "o250_v2250_P2500_G12500_K7500": (250, 2250, 2500, 12500, 7500, 3),
    # first held-out system of the learned-preconditioner protocol
    "o60_v300_P600_G1800_K900": (60, 300, 600, 1800, 900, 200),
}


def config_system(name: str, max_bytes: float = 64e9) -> System:
    """The named workload.  Refuses systems whose float64 Cholesky array
    (K n^2 doubles) exceeds max_bytes: the 2500-basis shape needs 375 GB
    (and 2 n^2 G K = 1.2e15 flops to form); ``make_device_system`` forms it
    on a GPU in slabs instead."""
    o, v, P, G, K, seed = CONFIGS[name]
    need = 8.0 * K * (o + v) ** 2
    if need > max_bytes:
        raise MemoryError(f"{name}: the Cholesky array takes {need / 1e9:.0f} GB "
                          f"(limit {max_bytes / 1e9:.0f} GB)")
    return make_system(o, v, P, G, K, seed)
