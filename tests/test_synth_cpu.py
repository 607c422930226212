"""The seeded input recipe: shapes, symmetry, ordering, ranges and the stated
distributions of the synthetic molecules (orbital energies, RI factors,
dipoles), determinism by seed, and unit-norm random states."""
import numpy as np
import pytest

from paper_2601_16949_b300 import synth


def test_shapes_symmetry_ordering_and_ranges():
    o, v, P = 7, 19, 11
    m = synth.molecule(o, v, P, seed=3)
    shapes = dict(eps_occ=(o,), eps_virt=(v,), B_ov=(P, o, v), B_oo=(P, o, o), B_vv=(P, v, v),
                  mu_oo=(3, o, o), mu_vv=(3, v, v), mu_0ov=(3, o, v))
    for k, shp in shapes.items():
        assert m[k].shape == shp and m[k].dtype == np.float64 and m[k].flags.c_contiguous, k
    for k in ("B_oo", "B_vv", "mu_oo", "mu_vv"):
        assert np.array_equal(m[k], np.swapaxes(m[k], -1, -2)), k
    assert np.all(np.diff(m["eps_occ"]) >= 0) and np.all(np.diff(m["eps_virt"]) >= 0)
    assert m["eps_occ"].min() >= -1.0 and m["eps_occ"].max() <= -0.3
    assert m["eps_virt"].min() >= 0.05 and m["eps_virt"].max() <= 2.0
    assert (m["nocc"], m["nvirt"], m["naux"]) == (o, v, P)


def test_distributions_match_the_recipe():
    """B^P_pq ~ N(0, 0.05^2 / naux); mu blocks ~ N(0, 0.5^2); <0|mu|ia> ~
    N(0, 0.3^2); means near zero (standard errors from the sample sizes)."""
    o, v, P = 16, 64, 256
    m = synth.molecule(o, v, P, seed=0)
    iu_v = np.triu_indices(v)
    cases = [
        (m["B_ov"].ravel(), 0.05 / np.sqrt(P)),
        (m["B_vv"][:, iu_v[0], iu_v[1]].ravel(), 0.05 / np.sqrt(P)),
        (m["mu_vv"][:, iu_v[0], iu_v[1]].ravel(), 0.5),
        (m["mu_0ov"].ravel(), 0.3),
    ]
    for x, sd in cases:
        n = x.size
        assert abs(x.mean()) < 5 * sd / np.sqrt(n)
        assert abs(x.std() / sd - 1.0) < 5 / np.sqrt(2 * n) + 1e-3


def test_seeded_and_reproducible():
    a = synth.molecule(3, 5, 4, seed=9)
    b = synth.molecule(3, 5, 4, seed=9)
    c = synth.molecule(3, 5, 4, seed=10)
    for k in ("eps_occ", "eps_virt", "B_ov", "B_oo", "B_vv", "mu_oo", "mu_vv", "mu_0ov"):
        assert np.array_equal(a[k], b[k])
        assert not np.array_equal(a[k], c[k])


def test_random_states_are_unit_norm_per_trajectory():
    c = synth.random_state(97, 4, seed=2)
    assert c.shape == (4, 97) and np.iscomplexobj(c)
    assert np.allclose(np.linalg.norm(c, axis=1), 1.0, atol=1e-14)
    assert np.array_equal(c, synth.random_state(97, 4, seed=2))


def test_rejects_empty_dimensions():
    with pytest.raises(ValueError):
        synth.molecule(0, 3, 3)
