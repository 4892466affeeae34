"""Seeded synthetic Kohn-Sham matrices (H, S) shared by the tests, the oracle checks and
the benchmark. This module holds input construction only: none of the solver's
arithmetic (no factorisation, no eigensolver, no occupation, no density matrix).

The paper's workloads are FHI-aims / DGDFT graphene Hamiltonians (arXiv:1705.11191,
Table 1) that are not available here; these decaying random matrices stand in for
them with the same shape: 8-15 basis functions per atom, an occupied fraction of 25 %
(within the 10-40 % the paper quotes for localized basis sets, sec. 2) and a
positive-definite overlap.

Recipe (all draws from numpy's PCG64 ``default_rng(seed)`` in this order):
  1. atom positions (1D chain: fixed spacing; 3D cluster: uniform in a cube, rejection
     sampling for a 2 bohr minimum separation);
  2. u  = rng.random((n, n))        -> S off-diagonal factors (upper triangle used);
  3. hd = rng.uniform(-1, 0.5, n)  -> H diagonal (onsite energies, Ha);
  4. g  = rng.standard_normal((n, n)) -> H off-diagonal noise (upper triangle used).
  With d_ij the distance between the atoms carrying basis functions i and j
  (0 on the same atom):
     O_ij = 0.3 exp(-d_ij/1.5) u_ij               (i != j, mirrored from i < j)
     H_ij = -0.5 exp(-d_ij/1.2) (1 + 0.1 g_ij)    (i != j, mirrored from i < j)
     S    = I + alpha O, alpha = 1, or, when lambda_min(I + O) < tau,
            alpha = (1 - tau) / (-lambda_min(O)) so that lambda_min(S) = tau exactly.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Problem", "chain_positions", "cluster_positions", "build", "cluster_problem", "chain_problem", "kpoint_problem",
           "basis_atoms", "WORKLOADS", "workload"]


@dataclasses.dataclass
class Problem:
    h: np.ndarray          # (n, n) float64, column-major (Fortran order)
    s: np.ndarray          # (n, n) float64, column-major
    n_electron: float
    n_state: int
    name: str
    lambda_min_s: float

    @property
    def n(self) -> int:
        return self.h.shape[0]


def chain_positions(n_atoms: int, spacing: float = 2.0) -> np.ndarray:
    x = np.zeros((n_atoms, 3))
    x[:, 0] = spacing * np.arange(n_atoms)
    return x


def cluster_positions(rng: np.random.Generator, n_atoms: int, density: float = 0.01,
                      min_sep: float = 2.0) -> np.ndarray:
    side = (n_atoms / density) ** (1.0 / 3.0)
    pos = np.zeros((n_atoms, 3))
    k = 0
    while k < n_atoms:
        p = rng.random(3) * side
        if k == 0 or np.min(np.sum((pos[:k] - p) ** 2, axis=1)) >= min_sep * min_sep:
            pos[k] = p
            k += 1
    return pos


def basis_atoms(n: int, per_atom: int) -> np.ndarray:
    """Atom index of each basis function: per_atom functions per atom, the last atom
    carrying the remainder."""
    return np.arange(n) // per_atom


def _lambda_min(o: np.ndarray) -> float:
    n = o.shape[0]
    if n <= 2048:
        return float(np.linalg.eigvalsh(o)[0])
    from scipy.sparse.linalg import eigsh
    w = eigsh(o, k=1, which="SA", tol=1e-12, return_eigenvectors=False)
    return float(w[0])


def build(rng: np.random.Generator, pos: np.ndarray, n: int, per_atom: int,
          tau: float = 1e-2, force_tau: bool = False):
    """Returns (H, S, lambda_min(S)) for the atom positions and basis layout."""
    atom = basis_atoms(n, per_atom)
    xyz = pos[atom]                                     # (n, 3)
    d = np.zeros((n, n))
    for c in range(3):
        diff = xyz[:, c][:, None] - xyz[:, c][None, :]
        d += diff * diff
    np.sqrt(d, out=d)
    u = rng.random((n, n))
    iu = np.triu_indices(n, 1) if n <= 4096 else None
    o = np.exp(-d / 1.5)
    o *= 0.3
    o *= u
    del u
    _mirror_upper(o)
    np.fill_diagonal(o, 0.0)
    hd = rng.uniform(-1.0, 0.5, n)
    g = rng.standard_normal((n, n))
    h = np.exp(-d / 1.2)
    h *= -0.5
    g *= 0.1
    g += 1.0
    h *= g
    del g, d
    _mirror_upper(h)
    h[np.diag_indices(n)] = hd
    lam_o = _lambda_min(o)
    alpha = 1.0
    if force_tau or 1.0 + lam_o < tau:
        alpha = (1.0 - tau) / (-lam_o)
    s = o
    s *= alpha
    s[np.diag_indices(n)] = 1.0
    del iu
    return (np.asfortranarray(h), np.asfortranarray(s), 1.0 + alpha * lam_o)


def _mirror_upper(a: np.ndarray, block: int = 2048) -> None:
    """a[j, i] = a[i, j] for i < j (the upper triangle is the authoritative draw)."""
    n = a.shape[0]
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        for c0 in range(r0, n, block):
            c1 = min(n, c0 + block)
            blk = a[r0:r1, c0:c1]
            if c0 == r0:
                up = np.triu(blk, 1)
                a[r0:r1, c0:c1] = up + up.T + np.diag(np.diag(blk))
            else:
                a[c0:c1, r0:r1] = blk.T


# The three real workloads by name: geometry, size, electrons, states, seed.
WORKLOADS = {
    "chain-n512": dict(geometry="chain", n=512, per_atom=8, n_atoms=64,
                       n_electron=256.0, n_state=512, seed=0),
    "cluster3d-n8192": dict(geometry="cluster", n=8192, per_atom=15, n_atoms=547,
                            n_electron=2048.0, n_state=1024, seed=1),
    "cluster3d-n16384": dict(geometry="cluster", n=16384, per_atom=15, n_atoms=1093,
                             n_electron=4096.0, n_state=2048, seed=2),
}


def cluster_problem(n: int, seed: int, per_atom: int = 15, tau: float = 1e-2,
                    force_tau: bool = False, n_state: int | None = None,
                    n_electron: float | None = None) -> Problem:
    """3D-cluster construction at any size n (used for the small parity cases)."""
    rng = np.random.default_rng(seed)
    n_atoms = math.ceil(n / per_atom)
    pos = cluster_positions(rng, n_atoms)
    h, s, lam = build(rng, pos, n, per_atom, tau=tau, force_tau=force_tau)
    ne = float(n // 4) if n_electron is None else float(n_electron)
    ns = max(1, int(math.ceil(ne / 2))) if n_state is None else int(n_state)
    return Problem(h, s, ne, ns, f"cluster3d-n{n}-seed{seed}", lam)


def chain_problem(n_atoms: int, per_atom: int, seed: int, n_electron: float,
                  n_state: int, tau: float = 1e-2) -> Problem:
    rng = np.random.default_rng(seed)
    n = n_atoms * per_atom
    pos = chain_positions(n_atoms)
    h, s, lam = build(rng, pos, n, per_atom, tau=tau)
    return Problem(h, s, float(n_electron), int(n_state), f"chain-n{n}-seed{seed}", lam)


def workload(name: str, tau: float | None = None) -> Problem:
    """One of WORKLOADS; tau forces lambda_min(S) = tau (the conditioning sweep)."""
    c = WORKLOADS[name]
    if c["geometry"] == "chain":
        return chain_problem(c["n_atoms"], c["per_atom"], c["seed"], c["n_electron"],
                             c["n_state"])
    rng = np.random.default_rng(c["seed"])
    pos = cluster_positions(rng, c["n_atoms"])
    h, s, lam = build(rng, pos, c["n"], c["per_atom"],
                      tau=1e-2 if tau is None else tau, force_tau=tau is not None)
    return Problem(h, s, c["n_electron"], c["n_state"], name, lam)


def kpoint_problem(n: int, kfrac, seed: int, per_atom: int = 15, density: float = 0.01,
                   tau: float = 1e-2) -> Problem:
    """Complex Hermitian k-point problem: n basis functions of a periodic cell (a random
    3D cluster of ceil(n/per_atom) atoms in a cube of side L repeated on a simple cubic
    lattice), 27 real lattice blocks H_R, O_R (R in {-1, 0, 1}^3) built with the decay
    rules above on the distances |x_a - x_b - R L|, H_{-R} = H_R^T, and
        H(k) = sum_R H_R e^{2 pi i kfrac . R},  S(k) = I + alpha sum_R O_R e^{2 pi i kfrac . R}
    (alpha chosen so that lambda_min(S(k)) >= tau). Draw order: positions, then for
    R in lexicographic order with R >= -R: u (n x n), g (n x n); then the H_0 diagonal."""
    rng = np.random.default_rng(seed)
    n_atoms = math.ceil(n / per_atom)
    pos = cluster_positions(rng, n_atoms, density=density)
    side = (n_atoms / density) ** (1.0 / 3.0)
    atom = basis_atoms(n, per_atom)
    xyz = pos[atom]
    kfrac = np.asarray(kfrac, dtype=float)
    hk = np.zeros((n, n), dtype=np.complex128)
    ok = np.zeros((n, n), dtype=np.complex128)
    cells = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    done = set()
    for R in cells:
        mR = tuple(-x for x in R)
        if mR in done:
            continue
        done.add(R)
        shift = np.array(R, dtype=float) * side
        d = np.zeros((n, n))
        for c in range(3):
            diff = xyz[:, c][:, None] - (xyz[:, c][None, :] + shift[c])
            d += diff * diff
        np.sqrt(d, out=d)
        u = rng.random((n, n))
        g = rng.standard_normal((n, n))
        oR = 0.3 * np.exp(-d / 1.5) * u
        hR = -0.5 * np.exp(-d / 1.2) * (1.0 + 0.1 * g)
        if R == (0, 0, 0):
            # the home cell block is symmetric: mirror the upper triangle, no self term
            oR = np.triu(oR, 1)
            oR = oR + oR.T
            hR = np.triu(hR, 1)
            hR = hR + hR.T
            ok += oR
            hk += hR
        else:
            ph = np.exp(2j * np.pi * float(kfrac @ np.array(R, dtype=float)))
            ok += oR * ph + oR.T * np.conj(ph)
            hk += hR * ph + hR.T * np.conj(ph)
    hd = rng.uniform(-1.0, 0.5, n)
    hk[np.diag_indices(n)] = hd
    hk = 0.5 * (hk + hk.conj().T)
    ok = 0.5 * (ok + ok.conj().T)
    lam = float(np.linalg.eigvalsh(ok)[0]) if n <= 4096 else float(
        __import__("scipy.sparse.linalg", fromlist=["eigsh"]).eigsh(ok, k=1, which="SA",
                                                                  return_eigenvectors=False)[0])
    alpha = 1.0 if 1.0 + lam >= tau else (1.0 - tau) / (-lam)
    sk = alpha * ok
    sk[np.diag_indices(n)] = 1.0
    ne = float(n // 4)
    return Problem(hk, sk, ne, max(1, int(math.ceil(ne / 2))), f"kpoint-n{n}-seed{seed}",
                   1.0 + alpha * lam)


# ---------------------------------------------------------------- batches of problems
# The two batches of the several-problem path (k-points of a periodic cell; uneven real
# problems). Draws come from numpy's PCG64 in the order stated; the elementwise
# construction and the lambda_min(S) rescale run with torch on `device` when one is given
# (a GPU makes the batch generation fast), else with numpy.

def _lam_min_torch(o, torch):
    return float(torch.linalg.eigvalsh(o)[0].item())


def kpoint_set(n: int, grid: int = 4, seed: int = 3, per_atom: int = 15, density: float = 0.01,
               tau: float = 1e-2, device=None):
    """Complex Hermitian problems H(k), S(k) of kpoint_problem(n, k, seed) for the
    Gamma-centred grid x grid x grid k-points k = (i, j, l) / grid (i slowest), built from one
    set of 27 real lattice blocks (the same draws as kpoint_problem). Returns a list of
    (kfrac, H, S, lambda_min(S)) with H, S torch complex128 tensors on `device` (row-major
    (n, n) tensors of the Hermitian matrices) and N_el = n // 4 per problem."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    rng = np.random.default_rng(seed)
    n_atoms = math.ceil(n / per_atom)
    pos = cluster_positions(rng, n_atoms, density=density)
    side = (n_atoms / density) ** (1.0 / 3.0)
    atom = basis_atoms(n, per_atom)
    xyz = torch.from_numpy(pos[atom]).to(dev)
    cells = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    done, blocks = set(), []
    for R in cells:
        mR = tuple(-x for x in R)
        if mR in done:
            continue
        done.add(R)
        shift = torch.tensor(R, dtype=torch.float64, device=dev) * side
        d = torch.cdist(xyz, xyz + shift[None, :], compute_mode="donot_use_mm_for_euclid_dist")
        u = torch.from_numpy(rng.random((n, n))).to(dev)
        g = torch.from_numpy(rng.standard_normal((n, n))).to(dev)
        oR = 0.3 * torch.exp(-d / 1.5) * u
        hR = -0.5 * torch.exp(-d / 1.2) * (1.0 + 0.1 * g)
        del d, u, g
        if R == (0, 0, 0):
            oR = torch.triu(oR, 1)
            oR = oR + oR.T
            hR = torch.triu(hR, 1)
            hR = hR + hR.T
        blocks.append((R, hR, oR))
    hd = torch.from_numpy(rng.uniform(-1.0, 0.5, n)).to(dev)
    out = []
    ks = [(i / grid, j / grid, l / grid) for i in range(grid) for j in range(grid)
          for l in range(grid)]
    for kf in ks:
        hk = torch.zeros((n, n), dtype=torch.complex128, device=dev)
        ok = torch.zeros((n, n), dtype=torch.complex128, device=dev)
        for R, hR, oR in blocks:
            if R == (0, 0, 0):
                hk += hR
                ok += oR
            else:
                ph = complex(np.exp(2j * np.pi * float(np.dot(kf, R))))
                hk += hR * ph + hR.T * ph.conjugate()
                ok += oR * ph + oR.T * ph.conjugate()
        hk.diagonal().copy_(hd.to(torch.complex128))
        hk = 0.5 * (hk + hk.conj().T)
        ok = 0.5 * (ok + ok.conj().T)
        lam = _lam_min_torch(ok, torch)
        alpha = 1.0 if 1.0 + lam >= tau else (1.0 - tau) / (-lam)
        sk = alpha * ok
        sk.diagonal().fill_(1.0)
        out.append((kf, hk, sk, 1.0 + alpha * lam))
    return out


def mixed_sizes(count: int = 200, seed: int = 4, lo: int = 256, hi: int = 4096):
    """n_i = round(exp(U(ln lo, ln hi))), i < count, from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(math.log(lo), math.log(hi), count)
    return [int(round(math.exp(v))) for v in x]


def cluster_problem_torch(n: int, seed: int, device, per_atom: int = 15, tau: float = 1e-2):
    """cluster_problem(n, seed) with the elementwise construction and the lambda_min(S)
    rescale on `device` (the same numpy draws in the same order). Returns
    (H, S, n_electron, n_state, lambda_min(S)) with H, S torch float64 (n, n) tensors
    (symmetric, so the row-major tensor is also the column-major matrix)."""
    import torch
    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    n_atoms = math.ceil(n / per_atom)
    pos = cluster_positions(rng, n_atoms)
    atom = basis_atoms(n, per_atom)
    xyz = torch.from_numpy(pos[atom]).to(dev)
    d = torch.cdist(xyz, xyz, compute_mode="donot_use_mm_for_euclid_dist")
    same = torch.from_numpy(atom[:, None] == atom[None, :]).to(dev)
    d = torch.where(same, torch.zeros_like(d), d)
    u = torch.from_numpy(rng.random((n, n))).to(dev)
    o = torch.triu(0.3 * torch.exp(-d / 1.5) * u, 1)
    del u
    o = o + o.T
    hd = torch.from_numpy(rng.uniform(-1.0, 0.5, n)).to(dev)
    g = torch.from_numpy(rng.standard_normal((n, n))).to(dev)
    h = torch.triu(-0.5 * torch.exp(-d / 1.2) * (1.0 + 0.1 * g), 1)
    del g, d
    h = h + h.T
    h.diagonal().copy_(hd)
    lam_o = _lam_min_torch(o, torch)
    alpha = 1.0
    if 1.0 + lam_o < tau:
        alpha = (1.0 - tau) / (-lam_o)
    s = alpha * o
    s.diagonal().fill_(1.0)
    ne = float(n // 4)
    return h, s, ne, max(1, int(math.ceil(ne / 2))), 1.0 + alpha * lam_o
