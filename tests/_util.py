"""Helpers shared by the tests: oracle reference runs and pulse conversion."""
import numpy as np

from oracle import rttda_oracle as orc


def oracle_pulse(p: dict) -> orc.Pulse:
    return orc.Pulse(kind=p["kind"], E0=p.get("E0", 0.0), omega=p.get("omega", 0.0), t0=p.get("t0", 0.0),
                     fwhm=p.get("fwhm", 1.0), beta=p.get("beta", 0.0), duration=p.get("duration", 0.0),
                     direction=tuple(p.get("direction", (0, 0, 1))))


def unit(d):
    d = np.asarray(d, dtype=np.float64)
    return d / np.linalg.norm(d)


def oracle_runs(mol, c_x, pulses, dt, nsteps, c0=None, integrator="rk4"):
    """Dense-oracle trajectories, one per pulse (each with its own M_d)."""
    A = orc.build_A(mol, c_x)
    run = orc.propagate if integrator == "rk4" else orc.propagate_sso
    out = []
    for t, p in enumerate(pulses):
        M = orc.build_M(*orc.dipole_along(mol, unit(p.get("direction", (0, 0, 1)))))
        out.append(run(A, M, oracle_pulse(p), None if c0 is None else c0[t], dt, nsteps))
    return out


def oracle_sigma(mol, c_x, pulses, c, t):
    """H(t) c per trajectory, dense oracle."""
    A = orc.build_A(mol, c_x)
    res = []
    for k, p in enumerate(pulses):
        M = orc.build_M(*orc.dipole_along(mol, unit(p.get("direction", (0, 0, 1)))))
        res.append(orc.sigma(A, M, orc.field(oracle_pulse(p), t), c[k]))
    return np.array(res)


def to_ri(c):
    return np.ascontiguousarray(np.stack([c.real, c.imag], axis=-1))
