"""Seeded synthetic RT-TDA inputs.

This module only draws random numbers. It holds none of the propagation
arithmetic, so the CPU oracle and the CUDA path can both take their inputs
from it without sharing any of the method.

Every draw uses numpy's PCG64 generator (``numpy.random.default_rng(seed)``),
so a seed gives the same arrays on every machine.

Distributions, all in atomic units:
  * occupied orbital energies  U[-1.0, -0.3] Ha, sorted ascending
  * virtual orbital energies   U[0.05, 2.0] Ha, sorted ascending
  * three-index factors B^P_pq N(0, 0.05^2 / naux).  B_oo and B_vv are
    symmetric in pq: the upper triangle (diagonal included) is drawn and
    mirrored.  B_ov is drawn independently.
  * MO dipole blocks mu_oo, mu_vv (x, y, z): symmetric, N(0, 0.5^2)
  * ground-to-singles dipole <0|mu|ia> (x, y, z): N(0, 0.3^2), independent.

Draw order: eps_occ, eps_virt, B_ov, B_oo, B_vv, mu_oo, mu_vv, mu_0ov.
"""
from __future__ import annotations

import numpy as np

__all__ = ["molecule", "molecule_device", "random_state", "FACTOR_SIGMA", "MU_SIGMA", "MU0_SIGMA"]

FACTOR_SIGMA = 0.05
MU_SIGMA = 0.5
MU0_SIGMA = 0.3


def _symmetric_block(rng: np.random.Generator, lead: int, n: int, scale: float) -> np.ndarray:
    """lead independent n x n symmetric matrices with N(0, scale^2) entries."""
    out = np.empty((lead, n, n), dtype=np.float64)
    iu = np.triu_indices(n)
    for p in range(lead):
        g = rng.standard_normal(len(iu[0])) * scale
        m = out[p]
        m[iu] = g
        m.T[iu] = g
    return out


def molecule(nocc: int, nvirt: int, naux: int, seed: int = 0,
             eps_occ_range=(-1.0, -0.3), eps_virt_range=(0.05, 2.0)) -> dict:
    """Draw one synthetic molecule (orbital energies, RI factors, dipoles).

    Returns a dict of C-contiguous float64 arrays:
      eps_occ [nocc], eps_virt [nvirt], B_ov [naux, nocc, nvirt],
      B_oo [naux, nocc, nocc], B_vv [naux, nvirt, nvirt],
      mu_oo [3, nocc, nocc], mu_vv [3, nvirt, nvirt], mu_0ov [3, nocc, nvirt].
    """
    if min(nocc, nvirt, naux) < 1:
        raise ValueError("nocc, nvirt and naux must be >= 1")
    rng = np.random.default_rng(seed)
    eps_occ = np.sort(rng.uniform(eps_occ_range[0], eps_occ_range[1], nocc))
    eps_virt = np.sort(rng.uniform(eps_virt_range[0], eps_virt_range[1], nvirt))
    fs = FACTOR_SIGMA / np.sqrt(naux)
    B_ov = rng.standard_normal((naux, nocc, nvirt)) * fs
    B_oo = _symmetric_block(rng, naux, nocc, fs)
    B_vv = _symmetric_block(rng, naux, nvirt, fs)
    mu_oo = _symmetric_block(rng, 3, nocc, MU_SIGMA)
    mu_vv = _symmetric_block(rng, 3, nvirt, MU_SIGMA)
    mu_0ov = rng.standard_normal((3, nocc, nvirt)) * MU0_SIGMA
    return dict(nocc=nocc, nvirt=nvirt, naux=naux,
                eps_occ=eps_occ, eps_virt=eps_virt,
                B_ov=B_ov, B_oo=B_oo, B_vv=B_vv,
                mu_oo=mu_oo, mu_vv=mu_vv, mu_0ov=mu_0ov)


def random_state(n: int, ntraj: int = 1, seed: int = 1, normalise: bool = True) -> np.ndarray:
    """Random complex amplitudes [ntraj, n] (unit norm per trajectory)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((ntraj, n)) + 1j * rng.standard_normal((ntraj, n))
    if normalise:
        c /= np.linalg.norm(c, axis=1, keepdims=True)
    return c


def molecule_device(nocc: int, nvirt: int, naux: int, seed: int = 0, device="cuda",
                    eps_occ_range=(-1.0, -0.3), eps_virt_range=(0.05, 2.0), slab: int = 128) -> dict:
    """Same distributions as molecule(), drawn on the GPU with torch's seeded
    Philox generator (a different stream than numpy's, so the values differ
    from molecule() for the same seed).  For molecules whose FP64 factors do
    not fit in host memory.  Returns contiguous float64 CUDA tensors with the
    same keys and layouts; symmetric blocks are drawn in slabs of P."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)

    def uni(n, lo, hi):
        return torch.sort(lo + (hi - lo) * torch.rand(n, generator=g, **f64)).values

    def sym(lead, n, scale):
        out = torch.empty((lead, n, n), **f64)
        for p0 in range(0, lead, slab):
            p1 = min(lead, p0 + slab)
            gm = torch.randn((p1 - p0, n, n), generator=g, **f64) * scale
            out[p0:p1] = torch.triu(gm) + torch.triu(gm, 1).transpose(1, 2)
            del gm
        return out

    fs = FACTOR_SIGMA / np.sqrt(naux)
    eps_occ = uni(nocc, *eps_occ_range)
    eps_virt = uni(nvirt, *eps_virt_range)
    B_ov = torch.randn((naux, nocc, nvirt), generator=g, **f64) * fs
    B_oo = sym(naux, nocc, fs)
    B_vv = sym(naux, nvirt, fs)
    mu_oo = sym(3, nocc, MU_SIGMA)
    mu_vv = sym(3, nvirt, MU_SIGMA)
    mu_0ov = torch.randn((3, nocc, nvirt), generator=g, **f64) * MU0_SIGMA
    return dict(nocc=nocc, nvirt=nvirt, naux=naux, eps_occ=eps_occ, eps_virt=eps_virt,
                B_ov=B_ov, B_oo=B_oo, B_vv=B_vv, mu_oo=mu_oo, mu_vv=mu_vv, mu_0ov=mu_0ov)
