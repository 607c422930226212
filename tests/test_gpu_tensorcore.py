"""GPU parity of the tcgen05 exchange paths (BF16 and BF16 hi/lo split)."""
import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import oracle_pulse, oracle_runs, oracle_sigma, to_ri, unit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PULSES = [
    dict(kind=1, E0=0.03, omega=0.7, direction=(0, 0, 1)),
    dict(kind=2, E0=0.05, omega=0.9, t0=2.0, fwhm=1.7, direction=(1, 0, 0)),
    dict(kind=4, E0=0.05, omega=1.1, duration=4.0, direction=(1, 1, 0)),
]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def _sigma_gpu(rb, prop, c, t):
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda")
    sd = torch.zeros_like(cd)
    rb.rttda_sigma(prop.h, cd.data_ptr(), t, sd.data_ptr(), 0)
    rb.rttda_sync(prop.h)
    s = sd.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1]


def _two_electron_part(mol, c_x, c):
    """(A - diag(e_a - e_i)) c: the part computed from the factors."""
    m0 = dict(mol)
    m0["eps_occ"] = np.zeros_like(mol["eps_occ"])
    m0["eps_virt"] = np.zeros_like(mol["eps_virt"])
    A2 = orc.build_A(m0, c_x)
    return np.array([A2 @ ck for ck in c])


# per-element error bounds relative to the two-electron scale, about 5-8x
# the largest error measured on these shapes (6e-6, 5e-4, 3e-3)
@pytest.mark.parametrize("prec,tol2e", [("bf16x3", 5e-5), ("bf16x2", 3e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("shape", [(3, 5, 7), (17, 70, 33), (64, 128, 40), (9, 192, 130)])
def test_sigma_tensorcore_matches_oracle(rb, prec, tol2e, shape):
    mol = synth.molecule(*shape, seed=12)
    c_x = 0.2
    prop = rb.Propagator(mol, c_x, prec)
    prop.set_field(PULSES)
    c = synth.random_state(prop.n, len(PULSES), seed=3)
    got = _sigma_gpu(rb, prop, c, 1.4)
    ref = oracle_sigma(mol, c_x, PULSES, c, 1.4)
    s2e = np.max(np.abs(_two_electron_part(mol, c_x, c)), axis=1)
    sall = np.max(np.abs(ref), axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    assert np.all(err <= tol2e * s2e + 2e-6 * sall), (err, s2e, sall)
    prop.close()


def test_bf16x3_exchange_only_matches_oracle_tightly(rb):
    """Isolate the exchange: zero Coulomb factors and orbital energies, no
    field; the hi/lo split must reproduce the FP64 exchange to ~1e-4."""
    mol = synth.molecule(32, 128, 64, seed=21)
    mol["B_ov"][:] = 0.0
    mol["eps_occ"][:] = 0.0
    mol["eps_virt"][:] = 0.0
    prop = rb.Propagator(mol, 1.0, "bf16x3")
    prop.set_field([dict(kind=0, E0=0.0)])
    c = synth.random_state(prop.n, 1, seed=4)
    got = _sigma_gpu(rb, prop, c, 0.5)
    A = orc.build_A(mol, 1.0)
    ref = A @ c[0]
    assert np.max(np.abs(got[0] - ref)) < 1e-4 * np.max(np.abs(ref))
    prop.close()


# relative dipole error after 400 steps, about 10x the measured error
# (7e-9, 1.5e-7, 3.1e-5 with the FP64-accurate observable)
@pytest.mark.parametrize("prec,dip_tol", [("bf16x3", 1e-7), ("bf16x2", 2e-6), ("bf16", 3e-4)])
def test_tensorcore_propagation_against_oracle(rb, prec, dip_tol):
    mol = synth.molecule(8, 64, 48, seed=5)
    pulses = [dict(kind=0, E0=1e-3, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 400)
    rb.rttda_sync(prop.h)
    refs = oracle_runs(mol, 0.2, pulses, 0.05, 400)
    for t, ref in enumerate(refs):
        d = ref.dipole - ref.dipole[0]
        rel = np.max(np.abs(dip[t] - ref.dipole)) / np.max(np.abs(d))
        assert rel < dip_tol, (prec, t, rel)
        assert np.max(np.abs(nrm[t] - ref.norm)) < 1e-9, (prec, t)
    prop.close()


def test_bf16x3_config2_sampled_rows(rb):
    """Full-size o=64, v=448, P=1536: sampled rows of one sigma against the
    oracle's element-wise rows."""
    mol = synth.molecule(64, 448, 1536, seed=0)
    pulses = [dict(kind=1, E0=0.01, omega=0.5, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    n = 1 + 64 * 448
    c = synth.random_state(n, 3, seed=11)
    rng = np.random.default_rng(1)
    rows = np.concatenate([[0, 1, n - 1], rng.choice(np.arange(2, n - 1), 21, replace=False)])
    Arows = orc.A_rows(mol, 0.2, rows)
    m0 = dict(mol)
    m0["eps_occ"] = np.zeros(64)
    m0["eps_virt"] = np.zeros(448)
    A2rows = orc.A_rows(m0, 0.2, rows)
    prop = rb.Propagator(mol, 0.2, "bf16x3")
    prop.set_field(pulses)
    got = _sigma_gpu(rb, prop, c, 0.9)
    prop.close()
    E = orc.field(orc.Pulse(kind=1, E0=0.01, omega=0.5), 0.9)
    for k, p in enumerate(pulses):
        Mrows = orc.M_rows(*orc.dipole_along(mol, unit(p["direction"])), rows)
        ref = Arows @ c[k] - E * (Mrows @ c[k])
        s2e = np.abs(A2rows) @ np.abs(c[k])
        sall = np.abs(Arows) @ np.abs(c[k]) + abs(E) * (np.abs(Mrows) @ np.abs(c[k]))
        err = np.abs(got[k, rows] - ref)
        assert np.all(err <= 2e-4 * s2e + 2e-6 * sall + 1e-300), (k, np.max(err / np.maximum(s2e, 1e-300)))


# per-element error bounds relative to the two-electron scale, about 5-8x
# the largest error measured on these shapes (6e-6, 5e-4, 3e-3)
@pytest.mark.parametrize("prec,tol2e", [("bf16x3", 5e-5), ("bf16x2", 3e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("shape", [(4, 70, 40), (8, 64, 48)])
def test_batched_sigma_with_tensorcore_coulomb(rb, prec, tol2e, shape):
    """Eight or more trajectories (16+ real columns) route the Coulomb passes
    through the tensor-core GEMM as well."""
    mol = synth.molecule(*shape, seed=31)
    pulses = [dict(kind=1, E0=0.01 * (k + 1), omega=0.3 + 0.1 * k, direction=(k % 3 == 0, k % 3 == 1, k % 3 == 2))
              for k in range(9)]
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field(pulses)
    c = synth.random_state(prop.n, len(pulses), seed=6)
    got = _sigma_gpu(rb, prop, c, 0.8)
    ref = oracle_sigma(mol, 0.2, pulses, c, 0.8)
    s2e = np.max(np.abs(_two_electron_part(mol, 0.2, c)), axis=1)
    sall = np.max(np.abs(ref), axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    assert np.all(err <= tol2e * s2e + 2e-6 * sall), (err, s2e, sall)
    prop.close()


WIDE_PLANS = ["160,3,32", "160,3,64", "192,2,32", "192,2,64",
              "64,2,32,t", "192,2,32,t", "256,2,32,t"]   # t: transposed (rows a, columns (col, i))


@pytest.mark.parametrize("prec,tol", [("bf16x2", 1e-2), ("bf16", 3e-2)])
def test_every_wide_plan_gives_the_same_exchange(rb, prec, tol, monkeypatch):
    """Exchange only (no Coulomb factors, orbital energies or field): each
    wide-M plan of the main contraction (tile width x row blocks x K tile,
    normal or transposed) computes the same sum up to FP32 summation order,
    and matches the FP64 exchange within the BF16 rounding of Z.  o=64 with
    3 trajectories gives 3 row blocks; v=128 is ragged for both tile widths;
    the transposed plans tile the 384 columns (col, i) by 64, 192 and 256
    (ragged)."""
    mol = synth.molecule(64, 128, 40, seed=31)
    mol["B_ov"][:] = 0.0
    mol["eps_occ"][:] = 0.0
    mol["eps_virt"][:] = 0.0
    c = synth.random_state(1 + 64 * 128, 3, seed=6)
    outs = []
    for plan in WIDE_PLANS:
        monkeypatch.setenv("RTTDA_WIDE_PLAN", plan)
        prop = rb.Propagator(mol, 1.0, prec)
        prop.set_field([dict(kind=0, E0=0.0)] * 3)
        info = rb.rttda_plan(prop.h)
        assert info["tuned"] == 3 and info["main_kernel"] == (4 if plan.endswith(",t") else 2)
        assert (info["main_bn"], info["main_mb"], info["main_kb"]) == tuple(int(x) for x in plan.split(",")[:3])
        outs.append(_sigma_gpu(rb, prop, c, 0.5))
        prop.close()
    A = orc.build_A(mol, 1.0)
    ref = np.array([A @ ck for ck in c])
    scale = np.max(np.abs(ref))
    for plan, got in zip(WIDE_PLANS, outs):
        assert np.max(np.abs(got - outs[0])) <= 2e-5 * scale, plan
        assert np.max(np.abs(got - ref)) <= tol * scale, plan


def test_wide_plan_tuner_times_every_candidate(rb, monkeypatch):
    monkeypatch.delenv("RTTDA_WIDE_PLAN", raising=False)
    monkeypatch.delenv("RTTDA_TUNE", raising=False)
    mol = synth.molecule(48, 96, 24, seed=8)
    prop = rb.Propagator(mol, 0.2, "bf16x2")
    prop.set_field(PULSES)
    info = rb.rttda_plan(prop.h)
    assert info["main_kernel"] in (2, 4) and info["tuned"] in (1, 2) and info["ntraj"] == 3
    if info["tuned"] == 1:
        assert info["ncand"] == 5 and all(t > 0 for t in info["tune_ms"])
    # the tuned plan is cached for the shape: a second handle reuses it
    p2 = rb.Propagator(mol, 0.2, "bf16x2")
    p2.set_field(PULSES)
    i2 = rb.rttda_plan(p2.h)
    assert i2["tuned"] == 2
    assert (i2["main_bn"], i2["main_mb"], i2["main_kb"], i2["main_splits"]) == \
        (info["main_bn"], info["main_mb"], info["main_kb"], info["main_splits"])
    c = synth.random_state(prop.n, 3, seed=2)
    assert np.array_equal(_sigma_gpu(rb, prop, c, 0.7), _sigma_gpu(rb, p2, c, 0.7))
    prop.close()
    p2.close()
    monkeypatch.setenv("RTTDA_WIDE_PLAN", "128,4,32")
    p3 = rb.Propagator(mol, 0.2, "bf16x2")
    with pytest.raises(rb.RTTDAError) as e:
        p3.set_field(PULSES)
    assert e.value.status == rb.E_ARG
    p3.close()


@pytest.mark.parametrize("prec", ["bf16x2", "bf16"])
def test_transposed_plan_for_one_trajectory(rb, prec, monkeypatch):
    """One trajectory: the C*o = 74 columns fill a transposed tile of 96
    (ragged); rows a = 150 span two 128-row blocks (ragged).  The transposed
    and the normal plans give the same sigma up to FP32 summation order, and
    both match the oracle within the BF16 tolerance."""
    mol = synth.molecule(37, 150, 20, seed=12)
    pulses = [dict(kind=2, E0=0.05, omega=0.9, t0=1.0, fwhm=1.5, direction=(0, 1, 0))]
    c = synth.random_state(1 + 37 * 150, 1, seed=9)
    outs = {}
    for plan in ("160,3,32", "96,2,32,t", "128,2,32,t"):
        monkeypatch.setenv("RTTDA_WIDE_PLAN", plan)
        prop = rb.Propagator(mol, 0.2, prec)
        prop.set_field(pulses)
        assert rb.rttda_plan(prop.h)["main_kernel"] == (4 if plan.endswith(",t") else 2)
        outs[plan] = _sigma_gpu(rb, prop, c, 0.8)
        prop.close()
    ref = oracle_sigma(mol, 0.2, pulses, c, 0.8)
    scale = np.max(np.abs(ref))
    tol = 1e-2 if prec == "bf16x2" else 3e-2
    for plan, got in outs.items():
        assert np.max(np.abs(got - outs["160,3,32"])) <= 2e-5 * scale, plan
        assert np.max(np.abs(got - ref)) <= tol * scale, plan


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
def test_z_build_tile_order_and_l2_policy_do_not_change_sigma(rb, prec, monkeypatch):
    """The one-plane Z build visits its tiles in slabs of row tiles
    (RTTDA_ZRUN tiles per CTA and column run; 0 = one slab) and stores Z
    under an L2 evict-first policy (RTTDA_ZHINT).  Neither changes any
    arithmetic: sigma is bitwise the same for every setting, here with
    768 row tiles (several slabs, the last one narrower) and a ragged last
    column tile, and it matches the oracle's rows of A and M_d."""
    mol = synth.molecule(64, 64, 1536, seed=5)
    c_x, t = 0.2, 0.9
    c = synth.random_state(1 + 64 * 64, len(PULSES), seed=8)
    out = {}
    for hint, run in ((1, 4), (0, 0), (1, 1), (0, 7)):
        monkeypatch.setenv("RTTDA_ZHINT", str(hint))
        monkeypatch.setenv("RTTDA_ZRUN", str(run))
        prop = rb.Propagator(mol, c_x, prec)
        prop.set_field(PULSES)
        out[(hint, run)] = _sigma_gpu(rb, prop, c, t)
        prop.close()
    base = out[(1, 4)]
    for k, v in out.items():
        assert np.array_equal(v, base), k
    n = 1 + 64 * 64
    rows = np.concatenate([[0, 1, n - 1], np.random.default_rng(3).choice(np.arange(2, n - 1), 13, replace=False)])
    Arows = orc.A_rows(mol, c_x, rows)
    m0 = dict(mol)
    m0["eps_occ"] = np.zeros_like(mol["eps_occ"])
    m0["eps_virt"] = np.zeros_like(mol["eps_virt"])
    A2rows = orc.A_rows(m0, c_x, rows)
    tol = {"bf16": 2e-2, "bf16x2": 3e-3}[prec]
    for k, pk in enumerate(PULSES):
        d = unit(pk["direction"])
        Mrows = orc.M_rows(*orc.dipole_along(mol, d), rows)
        E = orc.field(oracle_pulse(pk), t)
        ref = Arows @ c[k] - E * (Mrows @ c[k])
        s2e = np.abs(A2rows) @ np.abs(c[k])
        sall = np.abs(Arows) @ np.abs(c[k]) + abs(E) * (np.abs(Mrows) @ np.abs(c[k]))
        err = np.abs(base[k, rows] - ref)
        assert np.all(err <= tol * s2e + 2e-6 * sall), (prec, k, np.max(err / np.maximum(s2e, 1e-300)))


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
@pytest.mark.parametrize("cl", [2, 4])
@pytest.mark.parametrize("kb", [64, 32])
def test_clustered_main_contraction_is_bitwise_the_plain_one(rb, prec, cl, kb, monkeypatch):
    """The wide-M main contraction, K tile 64 or 32, in clusters of 2 or 4 CTAs (RTTDA_WIDE_CLUSTER;
    4 is the default where the plan allows it, 1 turns clusters off):
    each CTA loads 128/CL rows of every Z tile and multicasts them to the
    cluster, and a stage is refilled only after every CTA of the cluster has
    released it.  The tiles, their K order and every multiply-add are those
    of the plain kernel, so sigma and a short propagation are bitwise the
    same (four column tiles of 192, one row block, split-K), and sigma
    matches the oracle's rows."""
    # naux such that the plan's split-K count gives at most 132 units, so the
    # clustered grid keeps it (a re-chosen count would sum in another order)
    mol = synth.molecule(32, 768, 40 if kb == 64 else 20, seed=9)
    pulses = [dict(kind=4, E0=0.01 * (k + 1), omega=0.6, duration=6.0, direction=(0, 0, 1)) for k in range(4)]
    monkeypatch.setenv("RTTDA_WIDE_PLAN", f"192,2,{kb}")
    n = 1 + 32 * 768
    c = synth.random_state(n, len(pulses), seed=5)
    res, splits = {}, {}
    for clu in (1, cl):
        monkeypatch.setenv("RTTDA_WIDE_CLUSTER", str(clu))
        prop = rb.Propagator(mol, 0.2, prec)
        prop.set_field(pulses)
        plan = rb.rttda_plan(prop.h)
        assert (plan["main_kernel"], plan["main_bn"], plan["main_mb"], plan["main_kb"]) == (2, 192, 2, kb), plan
        assert plan["main_cluster"] == clu and plan["main_grid"] % clu == 0, plan
        splits[clu] = plan["main_splits"]
        sig = _sigma_gpu(rb, prop, c, 2.5)
        _, dip, nrm = prop.propagate(0.05, 6, c0=c)
        prop.close()
        res[clu] = (sig, dip, nrm)
    assert splits[1] == splits[cl], splits
    for a, b in zip(res[1], res[cl]):
        assert np.array_equal(a, b)
    rows = np.concatenate([[0, 1, n - 1], np.random.default_rng(4).choice(np.arange(2, n - 1), 9, replace=False)])
    Arows = orc.A_rows(mol, 0.2, rows)
    m0 = dict(mol)
    m0["eps_occ"] = np.zeros_like(mol["eps_occ"])
    m0["eps_virt"] = np.zeros_like(mol["eps_virt"])
    A2rows = orc.A_rows(m0, 0.2, rows)
    Mrows = orc.M_rows(*orc.dipole_along(mol, unit((0, 0, 1))), rows)
    tol = {"bf16": 2e-2, "bf16x2": 3e-3}[prec]
    for k, pk in enumerate(pulses):
        E = orc.field(oracle_pulse(pk), 2.5)
        ref = Arows @ c[k] - E * (Mrows @ c[k])
        s2e = np.abs(A2rows) @ np.abs(c[k])
        sall = np.abs(Arows) @ np.abs(c[k]) + abs(E) * (np.abs(Mrows) @ np.abs(c[k]))
        err = np.abs(res[cl][0][k, rows] - ref)
        assert np.all(err <= tol * s2e + 2e-6 * sall), (prec, k, np.max(err / np.maximum(s2e, 1e-300)))
