"""Continuous-batching server: results alone vs in the mix, admission by
footprint, cancellation and bounded waits."""
import time

import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import oracle_runs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


SPEC = dict(gamma=2e-2, wmin=0.2, wmax=2.5, nfreq=97)

CASES = [  # (nocc, nvirt, naux, prec, pulse, nsteps, seed)
    (6, 70, 40, "fp64", dict(kind=0, E0=1e-3, direction=(0, 0, 1)), 300, 1),
    (9, 64, 36, "bf16x2", dict(kind=4, E0=0.02, omega=0.9, duration=8.0, direction=(1, 0, 0)), 420, 2),
    (4, 130, 52, "bf16x3", dict(kind=0, E0=2e-3, direction=(0, 1, 0)), 250, 3),
    (12, 48, 30, "fp32", dict(kind=2, E0=0.03, omega=0.7, t0=3.0, fwhm=2.0, direction=(0, 1, 1)), 360, 4),
    (5, 40, 24, "fp64oz", dict(kind=3, E0=0.02, omega=0.8, t0=2.0, fwhm=2.5, beta=0.2, direction=(1, 0, 1)), 200, 5),
]


def _request(rb, case):
    o, v, P, prec, pulse, nsteps, seed = case
    mol = synth.molecule(o, v, P, seed=seed)
    return mol, rb.make_request(mol, 0.2, prec, pulse, 0.05, nsteps, **SPEC)


def _run_server(rb, cases, budget=32 << 30, max_active=4, chunk=64):
    srv = rb.rttda_server_create(budget, max_active, chunk)
    reqs = [_request(rb, c) for c in cases]
    ids = [rb.rttda_server_submit(srv, q) for _, q in reqs]
    out = []
    for rid, case in zip(ids, cases):
        rb.rttda_server_wait(srv, rid, 300.0)
        st, S, om, dip, lat = rb.rttda_server_poll(srv, rid, SPEC["nfreq"], case[5])
        assert st == rb.REQ_DONE, rb.rttda_last_error()
        out.append((S, om, dip, lat))
    stats = rb.rttda_server_stats_get(srv)
    rb.rttda_server_destroy(srv)
    return out, stats


def _standalone(rb, case):
    o, v, P, prec, pulse, nsteps, seed = case
    mol = synth.molecule(o, v, P, seed=seed)
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field([pulse])
    _, dip, _ = prop.propagate(0.05, nsteps, want_state=False)
    prop.close()
    om, S = rb.rttda_spectrum(dip[0], 0.05, pulse["E0"], SPEC["gamma"], SPEC["wmin"], SPEC["wmax"], SPEC["nfreq"])
    return S, om, dip[0]


def test_each_result_is_the_same_alone_and_in_the_mix(rb):
    mixed, stats = _run_server(rb, CASES)
    assert stats["completed"] == len(CASES) and stats["max_concurrent"] >= 2
    for k, case in enumerate(CASES):
        alone, _ = _run_server(rb, [case])
        S_mix, om_mix, dip_mix, _ = mixed[k]
        S_one, om_one, dip_one, _ = alone[0]
        assert np.array_equal(dip_mix, dip_one), case
        assert np.array_equal(S_mix, S_one), case
        # and identical to the plain (unserved) propagation + spectrum
        S_ref, om_ref, dip_ref = _standalone(rb, case)
        assert np.array_equal(dip_mix, dip_ref), case
        assert np.max(np.abs(S_mix - S_ref)) <= 1e-12 * np.max(np.abs(S_ref)), case


def test_served_fp64_request_matches_oracle(rb):
    case = CASES[0]
    (S, om, dip, lat), = _run_server(rb, [case])[0]
    o, v, P, prec, pulse, nsteps, seed = case
    mol = synth.molecule(o, v, P, seed=seed)
    ref = oracle_runs(mol, 0.2, [pulse], 0.05, nsteps)[0]
    assert np.max(np.abs(dip - ref.dipole)) < 1e-11
    S_ref = orc.spectrum(ref.dipole, 0.05, pulse["E0"], SPEC["gamma"],
                         orc.frequency_grid(SPEC["wmin"], SPEC["wmax"], SPEC["nfreq"]))
    assert np.max(np.abs(S - S_ref)) < 1e-9 * np.max(np.abs(S_ref))
    assert lat > 0


def test_admission_by_footprint_serialises_requests(rb):
    big = max(rb.rttda_estimate_bytes(c[0], c[1], c[2], 1, c[3], c[5]) for c in CASES)
    out, stats = _run_server(rb, CASES, budget=int(big * 1.2), max_active=4)
    assert stats["completed"] == len(CASES)
    assert stats["max_concurrent"] == 1
    assert stats["bytes_in_use"] == 0


def test_cancel_pending_and_bounded_wait(rb):
    big = max(rb.rttda_estimate_bytes(c[0], c[1], c[2], 1, c[3], 20000) for c in CASES)
    srv = rb.rttda_server_create(int(big * 1.2), 1, 64)
    long_case = (6, 70, 40, "fp64", dict(kind=0, E0=1e-3), 20000, 1)
    _, q0 = _request(rb, long_case)
    _, q1 = _request(rb, CASES[1])
    r0 = rb.rttda_server_submit(srv, q0)
    r1 = rb.rttda_server_submit(srv, q1)
    rb.rttda_server_cancel(srv, r1)                      # still pending behind r0
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_server_wait(srv, r0, 1e-3)              # host wait with a tiny limit
    assert e.value.status == rb.E_TIMEOUT
    rb.rttda_server_cancel(srv, r0)                      # stops after its chunk in flight
    rb.rttda_server_wait(srv, r0, 120.0)
    rb.rttda_server_wait(srv, r1, 120.0)
    assert rb.rttda_server_poll(srv, r0)[0] == rb.REQ_CANCELLED
    assert rb.rttda_server_poll(srv, r1)[0] == rb.REQ_CANCELLED
    st = rb.rttda_server_stats_get(srv)
    assert st["cancelled"] == 2 and st["bytes_in_use"] == 0
    rb.rttda_server_destroy(srv)


def test_request_larger_than_budget_fails_cleanly(rb):
    srv = rb.rttda_server_create(1 << 20, 2, 64)       # 1 MiB: nothing fits
    _, q = _request(rb, CASES[0])
    rid = rb.rttda_server_submit(srv, q)
    rb.rttda_server_wait(srv, rid, 30.0)
    assert rb.rttda_server_poll(srv, rid)[0] == rb.REQ_FAILED
    assert "budget" in rb.rttda_last_error()
    rb.rttda_server_destroy(srv)


def test_cancel_and_destroy_while_handles_are_being_created(rb):
    """Handles are created on the server's creator thread while the
    scheduler steps the active requests.  Requests cancelled right after
    submission (before or during their handle's creation) end CANCELLED and
    give their memory back; the others still complete; destroying the server
    with requests queued for creation returns (nothing left behind)."""
    srv = rb.rttda_server_create(32 << 30, 3, 50)
    reqs = [_request(rb, c) for c in CASES[:4]]
    ids = [rb.rttda_server_submit(srv, q) for _, q in reqs]
    for k in (1, 3):
        rb.rttda_server_cancel(srv, ids[k])
    for rid in ids:
        rb.rttda_server_wait(srv, rid, 300.0)
    states = [rb.rttda_server_poll(srv, rid)[0] for rid in ids]
    assert states[0] == rb.REQ_DONE and states[2] == rb.REQ_DONE, states
    assert states[1] in (rb.REQ_CANCELLED, rb.REQ_DONE) and states[3] in (rb.REQ_CANCELLED, rb.REQ_DONE), states
    st = rb.rttda_server_stats_get(srv)
    assert st["bytes_in_use"] == 0 and st["completed"] + st["cancelled"] == 4
    rb.rttda_server_destroy(srv)
    # destroy with work still queued: returns without waiting for it
    srv = rb.rttda_server_create(32 << 30, 2, 50)
    for _, q in [_request(rb, c) for c in CASES]:
        rb.rttda_server_submit(srv, q)
    t0 = time.time()
    rb.rttda_server_destroy(srv)
    assert time.time() - t0 < 120.0
