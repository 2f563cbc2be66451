"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds only the *construction* of test Hamiltonians.  It contains
none of the SP2 method's arithmetic (no spectral bounds, no scaling, no
squaring, no traces, no density matrix): those live separately in the FP64
oracle and in the CUDA library.

Every Hamiltonian is built as H = Q diag(eps) Q^T with

* Q  the orthogonal factor of a Householder QR of a seeded N(0,1) matrix
  (columns sign-fixed so that diag(R) > 0, which makes Q unique), and
* eps sorted occupied eigenvalues drawn uniformly from ``occ`` followed by
  sorted virtual eigenvalues drawn uniformly from ``virt``.

The paper's workloads are dense, orthonormal-basis, real symmetric H with a
HOMO-LUMO gap (Sec. 2, Eqs. 1-6).  The recipes below reproduce those shapes:
gapped spectra around mu = 0, dense randomly rotated eigenvectors.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "Hamiltonian",
    "gapped_hamiltonian",
    "uniform_random_symmetric",
    "batched_config",
    "network_config",
    "CONFIGS",
]


@dataclasses.dataclass
class Hamiltonian:
    """A generated Hamiltonian with its exact spectral data.

    H   : (N, N) float64, symmetric (symmetrised as (A + A^T)/2)
    Q   : (N, N) float64 orthogonal eigenvectors (columns), or None
    eps : (N,)  float64 eigenvalues matching the columns of Q (ascending), or None
    n_occ : number of occupied states (the lowest n_occ eigenvalues)
    """

    H: np.ndarray
    Q: Optional[np.ndarray]
    eps: Optional[np.ndarray]
    n_occ: int
    seed: int

    @property
    def N(self) -> int:
        return self.H.shape[0]

    def h32(self) -> np.ndarray:
        """H rounded to FP32 (the storage the GPU path receives)."""
        return np.ascontiguousarray(self.H.astype(np.float32))


def _haar_q(N: int, rng: np.random.Generator, device: str = "cpu") -> np.ndarray:
    """Orthogonal factor of the QR of a seeded Gaussian matrix, sign-fixed.

    The Gaussian matrix always comes from numpy's PCG64 stream so that both
    sides see the same numbers.  For large N the QR itself may run through
    torch on a CUDA device in FP64 (test tooling only, never the SP2 path).
    """
    G = rng.standard_normal((N, N))
    if device != "cpu":
        import torch

        Gt = torch.from_numpy(G).to(device=device, dtype=torch.float64)
        Qt, Rt = torch.linalg.qr(Gt)
        d = torch.sign(torch.diagonal(Rt))
        d[d == 0] = 1.0
        Qt = Qt * d[None, :]
        Q = Qt.cpu().numpy()
        del Gt, Qt, Rt
        return Q
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def _assemble(Q: np.ndarray, eps: np.ndarray, device: str = "cpu") -> np.ndarray:
    if device != "cpu":
        import torch

        Qt = torch.from_numpy(Q).to(device=device, dtype=torch.float64)
        et = torch.from_numpy(eps).to(device=device, dtype=torch.float64)
        Ht = (Qt * et[None, :]) @ Qt.T
        Ht = 0.5 * (Ht + Ht.T)
        H = Ht.cpu().numpy()
        del Qt, et, Ht
        return H
    H = (Q * eps[None, :]) @ Q.T
    return 0.5 * (H + H.T)


def gapped_hamiltonian(
    N: int,
    n_occ: int,
    occ: Sequence[float] = (-1.0, -0.05),
    virt: Sequence[float] = (0.05, 1.0),
    seed: int = 0,
    device: str = "cpu",
) -> Hamiltonian:
    """Dense gapped Hamiltonian H = Q diag(eps) Q^T.

    ``n_occ`` eigenvalues are uniform in ``occ``, ``N - n_occ`` uniform in
    ``virt``; with occ[1] < virt[0] the HOMO-LUMO gap is at least
    virt[0] - occ[1] and the zero-temperature density matrix is unique.
    ``device`` = "cuda" runs the FP64 QR and the assembly through torch on the
    GPU (same random numbers; used for the large sizes).
    """
    if not (0 <= n_occ <= N):
        raise ValueError("n_occ must be in [0, N]")
    rng = np.random.default_rng(seed)
    if device == "cpu":
        Q = _haar_q(N, rng, device)
        e_occ = np.sort(rng.uniform(occ[0], occ[1], n_occ))
        e_virt = np.sort(rng.uniform(virt[0], virt[1], N - n_occ))
        eps = np.concatenate([e_occ, e_virt])
        H = _assemble(Q, eps, device)
        return Hamiltonian(H=H, Q=Q, eps=eps, n_occ=n_occ, seed=seed)
    import torch

    G = rng.standard_normal((N, N))
    e_occ = np.sort(rng.uniform(occ[0], occ[1], n_occ))
    e_virt = np.sort(rng.uniform(virt[0], virt[1], N - n_occ))
    eps = np.concatenate([e_occ, e_virt])
    with torch.no_grad():
        Gt = torch.from_numpy(G).to(device=device, dtype=torch.float64)
        del G
        Qt, Rt = torch.linalg.qr(Gt)
        del Gt
        d = torch.sign(torch.diagonal(Rt))
        d[d == 0] = 1.0
        del Rt
        Qt.mul_(d[None, :])
        et = torch.from_numpy(eps).to(device=device, dtype=torch.float64)
        Ht = (Qt * et[None, :]) @ Qt.T
        Ht = 0.5 * (Ht + Ht.T)
        H = Ht.cpu().numpy()
        del Ht
        Q = Qt.cpu().numpy()
        del Qt
        torch.cuda.empty_cache()
    return Hamiltonian(H=H, Q=Q, eps=eps, n_occ=n_occ, seed=seed)


def uniform_random_symmetric(N: int, n_occ: int, seed: int = 0) -> Hamiltonian:
    """H_ij ~ U[-1, 1], symmetrised (the small test matrices of Figs. 2 and 5).

    The spectrum is not known in closed form here (Q, eps are None).
    """
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, (N, N))
    H = np.triu(A) + np.triu(A, 1).T
    return Hamiltonian(H=H, Q=None, eps=None, n_occ=n_occ, seed=seed)


def batched_config(count: int = 512, seed: int = 1, n_min: int = 64, n_max: int = 1024,
                   step: int = 32):
    """Sizes and gaps of the batched workload.

    Returns a list of (N, n_occ, gap, instance_seed).  N is uniform over
    {n_min, n_min+step, ..., n_max}; gap g ~ U[0.05, 0.3]; n_occ = N/2; the
    spectrum of instance i is U[-1, -g/2] U U[g/2, 1] with seed 1000 + i.
    """
    rng = np.random.default_rng(seed)
    choices = np.arange(n_min, n_max + 1, step)
    Ns = rng.choice(choices, size=count)
    gaps = rng.uniform(0.05, 0.3, size=count)
    return [(int(n), int(n) // 2, float(g), 1000 + i) for i, (n, g) in enumerate(zip(Ns, gaps))]


def batched_instance(N: int, n_occ: int, gap: float, seed: int, device: str = "cpu") -> Hamiltonian:
    return gapped_hamiltonian(N, n_occ, (-1.0, -gap / 2), (gap / 2, 1.0), seed, device)


def network_config(batch: int = 64, N: int = 2048, device: str = "cpu", first_seed: int = 2000):
    """Instances of the differentiable-network workload: the N=4096-style
    construction (eps in [-1,-0.05] U [0.05,1], half occupied) at size N,
    seed first_seed + i for instance i."""
    return [gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), first_seed + i, device)
            for i in range(batch)]


# The five workloads (names used by tests and the bench).
CONFIGS = {
    "n128_fp64": dict(N=128, n_occ=64, occ=(-1.0, -0.1), virt=(0.1, 1.0), seed=0),
    "n4096_split": dict(N=4096, n_occ=2048, occ=(-1.0, -0.05), virt=(0.05, 1.0), seed=0),
    "n16384_split": dict(N=16384, n_occ=8192, occ=(-2.0, -0.025), virt=(0.025, 2.0), seed=0),
}
