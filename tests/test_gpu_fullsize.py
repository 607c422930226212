"""Full-size parity on sampled outputs: the batched field-scan molecule
(nocc=128, nvirt=768, naux=3072, 32 sin^2 trajectories) in the launch
configuration the benchmark uses, one sigma checked row by row against the
oracle's element-wise rows of A and M_d."""
import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import to_ri, unit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fieldscan():
    mol = synth.molecule(128, 768, 3072, seed=0)
    gap = float(np.min(mol["eps_virt"][None, :] - mol["eps_occ"][:, None]))
    amps = np.exp(np.linspace(np.log(1e-3), np.log(5e-2), 16))
    pulses = [dict(kind=4, E0=float(a), omega=w, duration=400.0, direction=(0.0, 0.0, 1.0))
              for w in (gap, 0.5 * gap) for a in amps]
    return mol, pulses


@pytest.mark.parametrize("prec,tol", [("bf16", 2e-2), ("bf16x2", 2e-3), ("bf16x3", 2e-4)])
def test_fieldscan_sigma_sampled_rows(fieldscan, prec, tol):
    from paper_2601_16949_b300 import binding as rb
    mol, pulses = fieldscan
    T = len(pulses)
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field(pulses)
    n = prop.n
    c = synth.random_state(n, T, seed=21)
    t = 137.0
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda")
    sd = torch.zeros_like(cd)
    rb.rttda_sigma(prop.h, cd.data_ptr(), t, sd.data_ptr(), 0)
    rb.rttda_sync(prop.h)
    prop.close()
    s = sd.cpu().numpy()
    got = s[..., 0] + 1j * s[..., 1]
    rng = np.random.default_rng(2)
    rows = np.concatenate([[0, 1, n - 1], rng.choice(np.arange(2, n - 1), 9, replace=False)])
    Arows = orc.A_rows(mol, 0.2, rows)
    m0 = dict(mol)
    m0["eps_occ"] = np.zeros_like(mol["eps_occ"])
    m0["eps_virt"] = np.zeros_like(mol["eps_virt"])
    A2rows = orc.A_rows(m0, 0.2, rows)
    Mrows = orc.M_rows(*orc.dipole_along(mol, unit((0.0, 0.0, 1.0))), rows)
    for k in (0, 7, 15, 16, 31):
        E = orc.field(orc.Pulse(kind=4, E0=pulses[k]["E0"], omega=pulses[k]["omega"], duration=400.0), t)
        ref = Arows @ c[k] - E * (Mrows @ c[k])
        s2e = np.abs(A2rows) @ np.abs(c[k])
        sall = np.abs(Arows) @ np.abs(c[k]) + abs(E) * (np.abs(Mrows) @ np.abs(c[k]))
        err = np.abs(got[k, rows] - ref)
        assert np.all(err <= tol * s2e + 2e-6 * sall + 1e-300), (prec, k, np.max(err / np.maximum(s2e, 1e-300)))


class _DeviceSlices:
    """B[:, k, :] of a CUDA tensor [P][n][n], fetched on demand for the oracle."""

    def __init__(self, t):
        self.t = t

    def __getitem__(self, key):
        _, k, _ = key
        return self.t[:, k, :].cpu().numpy()


def test_large_system_sigma_sampled_rows():
    """nocc=256, nvirt=1536, naux=4096 (dim 393217; B_vv 9.7e9 elements),
    factors drawn on the GPU and passed by device pointer; one sigma with a
    CW field, sampled rows against the oracle's element-wise rows."""
    from paper_2601_16949_b300 import binding as rb
    mol = synth.molecule_device(256, 1536, 4096, seed=0)
    pulses = [dict(kind=1, E0=0.02, omega=0.5, direction=(0.0, 0.0, 1.0))]
    n = 1 + 256 * 1536
    c = synth.random_state(n, 1, seed=5)
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda")
    got = {}
    for prec in ("bf16x2", "bf16x3"):
        prop = rb.Propagator(mol, 0.2, prec)
        prop.set_field(pulses)
        sd = torch.zeros_like(cd)
        rb.rttda_sigma(prop.h, cd.data_ptr(), 0.7, sd.data_ptr(), 0)
        rb.rttda_sync(prop.h)
        prop.close()
        s = sd.cpu().numpy()
        got[prec] = s[0, :, 0] + 1j * s[0, :, 1]
    hmol = dict(nocc=256, nvirt=1536, naux=4096, eps_occ=mol["eps_occ"].cpu().numpy(),
                eps_virt=mol["eps_virt"].cpu().numpy(), B_ov=mol["B_ov"].cpu().numpy(),
                B_oo=_DeviceSlices(mol["B_oo"]), B_vv=_DeviceSlices(mol["B_vv"]))
    mu = {k: mol[k].cpu().numpy() for k in ("mu_oo", "mu_vv", "mu_0ov")}
    del mol
    torch.cuda.empty_cache()
    rng = np.random.default_rng(4)
    rows = np.concatenate([[0, 1, n - 1], rng.choice(np.arange(2, n - 1), 5, replace=False)])
    Arows = orc.A_rows(hmol, 0.2, rows)
    A2rows = Arows.copy()
    for r, k in enumerate(rows):
        if k > 0:
            i, a = divmod(k - 1, 1536)
            A2rows[r, k] -= hmol["eps_virt"][a] - hmol["eps_occ"][i]
    Mrows = orc.M_rows(*orc.dipole_along(dict(mu_oo=mu["mu_oo"], mu_vv=mu["mu_vv"], mu_0ov=mu["mu_0ov"]),
                                         (0.0, 0.0, 1.0)), rows)
    E = orc.field(orc.Pulse(kind=1, E0=0.02, omega=0.5), 0.7)
    ref = Arows @ c[0] - E * (Mrows @ c[0])
    s2e = np.abs(A2rows) @ np.abs(c[0])
    sall = np.abs(Arows) @ np.abs(c[0]) + abs(E) * (np.abs(Mrows) @ np.abs(c[0]))
    for prec, tol in (("bf16x2", 2e-3), ("bf16x3", 2e-4)):
        err = np.abs(got[prec][rows] - ref)
        assert np.all(err <= tol * s2e + 2e-6 * sall + 1e-300), (prec, np.max(err / np.maximum(s2e, 1e-300)))
