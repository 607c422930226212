"""Exchange built a few values of P at a time (Z chunks, capped by
RTTDA_ZCHUNK): every path accumulates the chunks' partial contractions and
gives the single-chunk sigma up to its own summation order, and the
oracle's within the path's tolerance.  Chunk counts leave a ragged last
chunk."""
import numpy as np
import pytest

from paper_2601_16949_b300 import synth
from tests._util import oracle_sigma, to_ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PULSES = [dict(kind=1, E0=0.03, omega=0.7, direction=(0, 0, 1)),
          dict(kind=2, E0=0.05, omega=0.9, t0=1.0, fwhm=1.5, direction=(1, 0, 0))]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def _sigma(rb, mol, prec, c, t, monkeypatch, zchunk=None, plan=None):
    if zchunk is None:
        monkeypatch.delenv("RTTDA_ZCHUNK", raising=False)
    else:
        monkeypatch.setenv("RTTDA_ZCHUNK", str(zchunk))
    if plan is None:
        monkeypatch.delenv("RTTDA_WIDE_PLAN", raising=False)
    else:
        monkeypatch.setenv("RTTDA_WIDE_PLAN", plan)
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field(PULSES)
    info = rb.rttda_plan(prop.h)
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda")
    sd = torch.zeros_like(cd)
    rb.rttda_sigma(prop.h, cd.data_ptr(), t, sd.data_ptr(), 0)
    torch.cuda.synchronize()
    prop.close()
    s = sd.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1], info


@pytest.mark.parametrize("prec,same,tol", [("fp64", 1e-13, 1e-13), ("fp32", 2e-6, 3e-6),
                                           ("bf16x2", 2e-5, 1e-2), ("bf16x3", 2e-5, 2e-4)])
def test_chunked_exchange_equals_one_chunk(rb, prec, same, tol, monkeypatch):
    mol = synth.molecule(7, 70, 13, seed=21)
    c = synth.random_state(1 + 7 * 70, len(PULSES), seed=4)
    one, i1 = _sigma(rb, mol, prec, c, 0.9, monkeypatch)
    four, i4 = _sigma(rb, mol, prec, c, 0.9, monkeypatch, zchunk=4)
    assert i1["z_chunk"] == 13 and i4["z_chunk"] == 4
    ref = oracle_sigma(mol, 0.2, PULSES, c, 0.9)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(four - one)) <= same * scale
    assert np.max(np.abs(four - ref)) <= tol * scale


@pytest.mark.parametrize("plan", ["160,3,32", "96,2,32,t"])
def test_chunked_exchange_on_each_wide_orientation(rb, plan, monkeypatch):
    """BF16X2 with both orientations of the wide main contraction over
    three chunks (5 + 5 + 3 values of P)."""
    mol = synth.molecule(7, 70, 13, seed=22)
    c = synth.random_state(1 + 7 * 70, len(PULSES), seed=5)
    one, _ = _sigma(rb, mol, "bf16x2", c, 0.4, monkeypatch, plan=plan)
    three, info = _sigma(rb, mol, "bf16x2", c, 0.4, monkeypatch, zchunk=5, plan=plan)
    assert info["z_chunk"] == 5 and info["main_kernel"] == (4 if plan.endswith(",t") else 2)
    ref = oracle_sigma(mol, 0.2, PULSES, c, 0.4)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(three - one)) <= 2e-5 * scale
    assert np.max(np.abs(three - ref)) <= 1e-2 * scale
