"""Guard bands around every buffer the library writes for its caller.

Each output lives in the middle of a larger allocation whose head and tail
hold a canary bit pattern (a NaN payload no computation produces); after the
call the pattern must be intact and the output itself fully written.  This
stands in for a memory checker on the caller-visible writes: device outputs
of rttda_sigma, rttda_propagate_device and rttda_coulomb_noalloc, and host
outputs of rttda_propagate, in every precision and on ragged shapes."""
import ctypes as ct

import numpy as np
import pytest

from paper_2601_16949_b300 import synth
from tests._util import to_ri

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GUARD = 4096                   # words on each side
PATTERN = 0x7FF4DEADBEEF1234   # a signalling-NaN bit pattern
PRECS = ["fp64", "fp32", "bf16", "bf16x3", "bf16x2", "fp64oz"]
SHAPES = [(1, 1, 1), (5, 37, 19), (9, 130, 21)]
PULSES = [dict(kind=4, E0=0.05, omega=0.9, duration=3.0, direction=(1, 0, 0)),
          dict(kind=0, E0=0.02, direction=(0, 0, 1))]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def _dev(n):
    buf = torch.empty(n + 2 * GUARD, dtype=torch.float64, device="cuda")
    buf.view(torch.int64).fill_(PATTERN)
    return buf, buf[GUARD:GUARD + n]


def _dev_intact(buf, n):
    w = buf.view(torch.int64)
    return bool((w[:GUARD] == PATTERN).all()) and bool((w[GUARD + n:] == PATTERN).all())


def _dev_written(view):
    return not bool((view.view(torch.int64) == PATTERN).any())


def _host(n):
    buf = np.full(n + 2 * GUARD, PATTERN, dtype=np.uint64).view(np.float64)
    return buf, buf[GUARD:GUARD + n]


def _host_intact(buf, n):
    w = buf.view(np.uint64)
    return bool(np.all(w[:GUARD] == PATTERN)) and bool(np.all(w[GUARD + n:] == PATTERN))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_outputs_stay_inside_their_buffers(rb, prec, shape):
    mol = synth.molecule(*shape, seed=6)
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field(PULSES)
    T, n = len(PULSES), prop.n
    nsteps = 7
    # sigma (device)
    c = synth.random_state(n, T, seed=3)
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda").reshape(-1)
    sbuf, sv = _dev(T * n * 2)
    rb.rttda_sigma(prop.h, cd.data_ptr(), 0.4, sv.data_ptr(), 0)
    torch.cuda.synchronize()
    assert _dev_intact(sbuf, T * n * 2) and _dev_written(sv)
    # propagate (device buffers)
    cbuf, cv = _dev(T * n * 2)
    dbuf, dv = _dev(T * (nsteps + 1))
    nbuf, nv = _dev(T * (nsteps + 1))
    rb.rttda_propagate_device(prop.h, 0, 0.05, nsteps, cv.data_ptr(), dv.data_ptr(), nv.data_ptr(), 0)
    torch.cuda.synchronize()
    for buf, view, m in ((cbuf, cv, T * n * 2), (dbuf, dv, T * (nsteps + 1)), (nbuf, nv, T * (nsteps + 1))):
        assert _dev_intact(buf, m) and _dev_written(view)
    # propagate (host buffers)
    hc, hcv = _host(T * n * 2)
    hd, hdv = _host(T * (nsteps + 1))
    hn, hnv = _host(T * (nsteps + 1))
    addr = lambda a: a.ctypes.data_as(ct.c_void_p).value
    rb.rttda_propagate_ptr(prop.h, 0, 0.05, nsteps, addr(hcv), addr(hdv), addr(hnv))
    for buf, view, m in ((hc, hcv, T * n * 2), (hd, hdv, T * (nsteps + 1)), (hn, hnv, T * (nsteps + 1))):
        assert _host_intact(buf, m) and not np.any(view.view(np.uint64) == PATTERN)
    # the device and host runs agree
    assert np.array_equal(dv.cpu().numpy(), hdv)
    prop.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 40, 23)])
def test_noalloc_coulomb_output_stays_inside_its_buffer(rb, shape):
    o, v, P = shape
    mol = synth.molecule(o, v, P, seed=2)
    n = 1 + o * v
    B = torch.tensor(mol["B_ov"].reshape(P, o * v), dtype=torch.float64, device="cuda")
    c = synth.random_state(n, 3, seed=5)
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda").reshape(-1)
    obuf, ov_ = _dev(3 * n * 2)
    rb.rttda_coulomb_noalloc(o, v, P, B.data_ptr(), cd.data_ptr(), 3, ov_.data_ptr(), 0)
    torch.cuda.synchronize()
    assert _dev_intact(obuf, 3 * n * 2) and _dev_written(ov_)
