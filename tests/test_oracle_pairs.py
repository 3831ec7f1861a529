"""Pins of the oracle's pair-product kinematics (Sec. 1, Eq. pTotal and
Eq. Lorentz): each collision makes an electron and a positron that carry the
photons' total energy and momentum, sit on the mass shell, and, seen from the
centre-of-mass frame, fly apart back to back along a random direction.  The
pins check conservation, the mass shell, the rest-frame case, the paper's own
velocity-addition formula (an independent route to the same velocities), the
threshold, and the direction draw's uniformity."""
import math

import numpy as np
import pytest

import oracle

MEC2 = 0.51099895000


def beam(E, d):
    d = np.asarray(d, dtype=np.float64).reshape(-1, 3)
    d = d / np.linalg.norm(d, axis=1)[:, None]
    n = len(d)
    z = np.zeros(n)
    return {"px": z, "py": z, "pz": z, "dx": d[:, 0].copy(), "dy": d[:, 1].copy(),
            "dz": d[:, 2].copy(), "E": np.asarray(E, dtype=np.float64), "w": np.ones(n)}


def random_pairs(n, seed):
    rng = np.random.default_rng(seed)
    Ea = rng.lognormal(math.log(5.0), 0.8, n)
    Eb = rng.lognormal(math.log(5.0), 0.8, n)
    da = rng.normal(size=(n, 3)) * [0.3, 0.3, 1.0] + [0, 0, 2.0]
    db = rng.normal(size=(n, 3)) * [0.3, 0.3, 1.0] - [0, 0, 2.0]
    a, b = beam(Ea, da), beam(Eb, db)
    i = rng.integers(0, n, n)
    j = rng.integers(0, n, n)  # a photon of b other than i's partner index
    cs = a["dx"][i] * b["dx"][j] + a["dy"][i] * b["dy"][j] + a["dz"][i] * b["dz"][j]
    keep = (Ea[i] * Eb[j] * (1 - cs) / (2 * MEC2 ** 2) > 1.0 + 1e-6) & (i != j)
    return a, b, np.stack([i[keep], j[keep]], axis=1).astype(np.uint32)


def test_conservation_and_mass_shell():
    a, b, hits = random_pairs(4000, 1)
    assert len(hits) > 1000
    out = oracle.pair_products(a, b, hits, seed=7)
    i, j = hits[:, 0], hits[:, 1]
    E = a["E"][i] + b["E"][j]
    P = (a["E"][i][:, None] * np.stack([a["dx"], a["dy"], a["dz"]], 1)[i]
         + b["E"][j][:, None] * np.stack([b["dx"], b["dy"], b["dz"]], 1)[j])
    np.testing.assert_allclose(out[:, 0] + out[:, 4], E, rtol=1e-12)
    assert np.all(np.abs(out[:, 1:4] + out[:, 5:8] - P) <= 1e-12 * E[:, None])
    for o in (0, 4):
        m2 = out[:, o] ** 2 - np.sum(out[:, o + 1:o + 4] ** 2, axis=1)
        assert np.all(np.abs(m2 - MEC2 ** 2) <= 1e-12 * out[:, o] ** 2)
        assert (out[:, o] >= MEC2 * (1 - 1e-12)).all()


def test_rest_frame_head_on():
    # equal energies, exactly head on: the CoM is at rest, each particle has the
    # photon energy, and the electron flies along the drawn direction
    E = 3.0
    a, b = beam([E], [[0, 0, 1]]), beam([E], [[0, 0, -1]])
    out = oracle.pair_products(a, b, np.array([[0, 0]], np.uint32), seed=11)[0]
    n = oracle.com_direction(11, 0, 0)
    p = math.sqrt(E * E - MEC2 * MEC2)
    assert out[0] == pytest.approx(E, rel=1e-15) and out[4] == pytest.approx(E, rel=1e-15)
    np.testing.assert_allclose(out[1:4], p * n, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(out[5:8], -p * n, rtol=1e-14, atol=1e-15)


def test_paper_velocity_addition_gives_the_same_velocities():
    # Eq. Lorentz with its garbled perpendicular part read as beta'_perp =
    # beta' - beta'_par: beta = (bc + b'_par + b'_perp sqrt(1 - bc^2)) / (1 + b'.bc)
    a, b, hits = random_pairs(3000, 2)
    out = oracle.pair_products(a, b, hits, seed=3)
    for k, (ii, jj) in enumerate(hits[:400]):
        E1, E2 = a["E"][ii], b["E"][jj]
        d1 = np.array([a["dx"][ii], a["dy"][ii], a["dz"][ii]])
        d2 = np.array([b["dx"][jj], b["dy"][jj], b["dz"][jj]])
        E, P = E1 + E2, E1 * d1 + E2 * d2
        bc = P / E
        M2 = 2 * E1 * E2 * (1 - d1 @ d2)
        bprime = math.sqrt(1 - 4 * MEC2 ** 2 / M2)  # CoM speed of each particle
        n = oracle.com_direction(3, int(ii), int(jj))
        for sign, o in ((1, 0), (-1, 4)):
            bp = sign * bprime * n
            u = bc / np.linalg.norm(bc)
            par = (bp @ u) * u
            perp = bp - par
            beta = (bc + par + perp * math.sqrt(1 - bc @ bc)) / (1 + bp @ bc)
            np.testing.assert_allclose(out[k, o + 1:o + 4] / out[k, o], beta, rtol=1e-9,
                                       atol=1e-12)
    assert len(hits) > 400


def test_below_threshold_is_refused():
    a, b = beam([0.3], [[0, 0, 1]]), beam([0.3], [[0, 0, -1]])  # s = 0.34 < 1
    with pytest.raises(ValueError):
        oracle.pair_products(a, b, np.array([[0, 0]], np.uint32), seed=1)


def test_direction_draw_is_uniform_on_the_sphere():
    n = np.array([oracle.com_direction(5, i, 1000 + i) for i in range(20000)])
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, rtol=0, atol=4e-16)
    assert np.all(np.abs(n.mean(axis=0)) < 0.03)  # 4 sigma for 20000 draws
    np.testing.assert_allclose((n ** 2).mean(axis=0), 1 / 3, atol=0.012)
    # the draw is a function of (seed, i, j) alone
    assert np.array_equal(oracle.com_direction(5, 3, 1003), n[3])
    assert not np.array_equal(oracle.com_direction(6, 3, 1003), n[3])
