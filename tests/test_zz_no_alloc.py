"""The allocation-free Coulomb entry point, checked against rttda_sigma and
against the oracle's explicit matrix.

rttda_coulomb_noalloc serves callers that may not allocate GPU memory while
they run (their device memory belongs to their own pool or has a fixed
budget).  Its scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has run every
other test already; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import to_ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _coulomb_only_molecule(o, v, P, seed):
    """A molecule whose sigma is the Coulomb term alone: no orbital-energy
    differences and no exchange factors (the field is a kick, so E(t>0)=0)."""
    mol = synth.molecule(o, v, P, seed=seed)
    mol["eps_occ"][:] = 0.0
    mol["eps_virt"][:] = 0.0
    mol["B_oo"][:] = 0.0
    mol["B_vv"][:] = 0.0
    return mol


def test_noalloc_coulomb_matches_sigma_on_two_calls():
    from paper_2601_16949_b300 import binding as rb
    o, v, P = 7, 40, 23
    mol = _coulomb_only_molecule(o, v, P, seed=17)
    pulses = [dict(kind=0, E0=1e-3, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    prop = rb.Propagator(mol, 0.2, "fp64")
    prop.set_field(pulses)
    n = prop.n
    A = orc.build_A(mol, 0.2)
    B = torch.tensor(mol["B_ov"].reshape(P, o * v), dtype=torch.float64, device="cuda")
    for call in range(2):
        c = synth.random_state(n, 3, seed=30 + call)
        cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda")
        ref = torch.zeros_like(cd)
        rb.rttda_sigma(prop.h, cd.data_ptr(), 1.0, ref.data_ptr(), 0)
        rb.rttda_sync(prop.h)
        out = torch.full_like(cd, float("nan"))
        torch.cuda.synchronize()
        rb.rttda_coulomb_noalloc(o, v, P, B.data_ptr(), cd.data_ptr(), 3, out.data_ptr(), 0)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) <= 1e-13 * np.max(np.abs(r)), call
        # the oracle: with zero orbital energies and exchange factors, A is
        # the Coulomb block 2 B_ov^T B_ov alone (ground row and column zero)
        want = (A @ c.T).T
        got = g[..., 0] + 1j * g[..., 1]
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want)), call
    prop.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2601_16949_b300 import binding as rb
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_coulomb_noalloc(2, 2, 1 << 19, p, p, 2, p, 0)   # 2^19 * 2 * 2 > 2^20
    assert e.value.status == rb.E_ARG
    assert "exceeds" in str(e.value)
