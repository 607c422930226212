"""A handle keeps its executable step graph between calls and gives it each
call's parameters by a graph update.  Every call must therefore behave like
the same call on a fresh handle, bit for bit, when these change between calls
on one handle: the time step, the step count, the time base of a resume, the
batch (number of trajectories, pulses), the integrator and the output
buffers.  The same sequence with a new graph per call (RTTDA_GRAPH_CACHE=0)
gives the same bits."""
import numpy as np
import pytest

from paper_2601_16949_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P1 = [dict(kind=4, E0=0.05, omega=0.9, duration=3.0, direction=(1, 0, 0)),
      dict(kind=0, E0=0.02, direction=(0, 0, 1))]
P2 = [dict(kind=2, E0=0.03, omega=0.7, t0=1.0, fwhm=1.5, direction=(0, 1, 0))]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def _fresh(rb, mol, prec, pulses, dt, nsteps, integrator="rk4"):
    p = rb.Propagator(mol, 0.2, prec, integrator=integrator)
    p.set_field(pulses)
    out = p.propagate(dt, nsteps)
    p.close()
    return out


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("prec", ["fp64", "bf16x2"])
@pytest.mark.parametrize("cache", ["1", "0"])
def test_each_call_on_one_handle_equals_a_fresh_handle(rb, prec, cache, monkeypatch):
    monkeypatch.setenv("RTTDA_GRAPH_CACHE", cache)
    # one plan for every handle, so that the BF16X2 sums are in the same order
    monkeypatch.setenv("RTTDA_WIDE_PLAN", "96,2,32,t")
    mol = synth.molecule(5, 37, 19, seed=8)
    a = rb.Propagator(mol, 0.2, prec)
    a.set_field(P1)
    r1 = a.propagate(0.05, 12)
    r2 = a.propagate(0.04, 7)                 # new time step and step count
    c3, d3, n3 = a.resume(0.04, 5)            # time base 7 dt
    a.set_field(P2)                           # new batch: one trajectory
    r4 = a.propagate(0.03, 9)
    rb.rttda_set_integrator(a.h, "sso")
    r5 = a.propagate(0.05, 6)
    a.close()

    assert _same(r1, _fresh(rb, mol, prec, P1, 0.05, 12))
    assert _same(r2, _fresh(rb, mol, prec, P1, 0.04, 7))
    c, d, n = _fresh(rb, mol, prec, P1, 0.04, 12)
    assert np.array_equal(c3, c)
    assert np.array_equal(d3, d[:, 7:]) and np.array_equal(n3, n[:, 7:])
    assert _same(r4, _fresh(rb, mol, prec, P2, 0.03, 9))
    assert _same(r5, _fresh(rb, mol, prec, P2, 0.05, 6, integrator="sso"))


def test_device_calls_on_new_buffers_and_streams(rb, monkeypatch):
    """rttda_propagate_device twice on one handle, the second time into other
    device buffers and on another stream: the second call's outputs land in
    its own buffers and equal the first call's."""
    monkeypatch.delenv("RTTDA_GRAPH_CACHE", raising=False)
    mol = synth.molecule(4, 20, 11, seed=3)
    p = rb.Propagator(mol, 0.2, "fp64")
    p.set_field(P1)
    T, n, K = 2, 1 + 4 * 20, 10
    outs = []
    for k in range(2):
        stream = torch.cuda.Stream()
        c = torch.zeros((T, n, 2), dtype=torch.float64, device="cuda")
        d = torch.zeros((T, K + 1), dtype=torch.float64, device="cuda")
        r = torch.zeros_like(d)
        rb.rttda_propagate_device(p.h, 0, 0.05, K, c.data_ptr(), d.data_ptr(), r.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        outs.append((c.cpu().numpy(), d.cpu().numpy(), r.cpu().numpy()))
    p.close()
    assert _same(outs[0], outs[1])
    assert np.all(outs[1][2] > 0.0)           # the second call's norms were written
