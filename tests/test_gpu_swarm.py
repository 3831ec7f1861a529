"""The IP regime on the GPU (trilens_swarm_mark / _count / _expand, then the
exact path on the real photons) against the FP64 oracle (Sec. 2.2): every
real-photon hit as (MP, photon in swarm, MP, photon in swarm), bit for bit --
small swarm beams over two steps, a point photon crossing a 20000-photon swarm,
weight-1 MPs (the single-photon path), and the full-size 2 x 16384-MP workload
(1.6M real photons per beam) on sampled MP pairs, including pairs whose MPs
were not marked (the oracle must find no hit there)."""
import math

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MEC2 = 0.51099895000


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_ip_hits(a, b, h_a, h_b, dt, kappa, steps):
    """Real-photon hits per step, mapped to (i, k, j, l) and sorted; and the marks."""
    A, B = binding.to_device(a), binding.to_device(b)
    sp = binding.swarm_split(A, B, h_a, h_b, dt, kappa, steps[0], len(steps))
    oa, ka = sp["owner_a"].cpu().numpy(), sp["k_a"].cpu().numpy()
    ob, kb = sp["owner_b"].cpu().numpy(), sp["k_b"].cpu().numpy()
    out = {}
    with binding.Collider(sp["a"], sp["b"], dt, kappa) as col:
        for k in steps:
            h, _ = col.step_hits(k)
            q = np.stack([oa[h[:, 0]], ka[h[:, 0]], ob[h[:, 1]], kb[h[:, 1]]], axis=1)
            out[k] = q[np.lexsort(q.T[::-1])].astype(np.uint32)
    return out, sp


def swarm_beams(n, seed, wmax):
    wl = synth.tiny_headon(n=n, seed=seed)
    a, b = synth.beams(wl)
    rng = np.random.default_rng(seed)
    a["w"] = rng.integers(1, wmax + 1, n).astype(np.float64)
    b["w"] = rng.integers(1, wmax + 1, n).astype(np.float64)
    return wl, a, b


@pytest.mark.parametrize("seed,h_a,h_b", [(41, 0.4, 0.4), (42, 1.5, 0.2), (43, 0.0, 0.8)])
def test_small_swarms_bit_exact(seed, h_a, h_b):
    wl, a, b = swarm_beams(80, seed, 6)
    got, sp = gpu_ip_hits(a, b, h_a, h_b, wl.dt, wl.kappa, [0, 1])
    total = 0
    for k in (0, 1):
        ref = oracle.ip_bruteforce(a, b, h_a, h_b, k, wl.dt, wl.kappa)
        assert np.array_equal(got[k], ref), (k, len(got[k]), len(ref))
        total += len(ref)
    assert total > 100
    # every MP of an oracle hit is marked
    ma, mb = sp["mark_a"].cpu().numpy(), sp["mark_b"].cpu().numpy()
    for k in (0, 1):
        ref = oracle.ip_bruteforce(a, b, h_a, h_b, k, wl.dt, wl.kappa)
        assert ma[ref[:, 0]].all() and mb[ref[:, 2]].all()


def one_mp(p, d, E, w):
    f = lambda x: np.array([float(x)])  # noqa: E731
    return {"px": f(p[0]), "py": f(p[1]), "pz": f(p[2]), "dx": f(d[0]), "dy": f(d[1]),
            "dz": f(d[2]), "E": f(E), "w": f(w)}


def test_point_photon_through_a_swarm():
    w, h, r = 20000, 1.0, 0.2
    s = 1.0 * 1.0 * 2.0 / (2 * MEC2 * MEC2)
    kappa = math.pi * r * r / (1e12 * oracle.sigma(s))
    a = one_mp((0, 0, 0), (0, 0, 1), 1.0, w)
    b = one_mp((0, 0, 5.0), (0, 0, -1), 1.0, 1)
    got, _ = gpu_ip_hits(a, b, h, 0.0, 20.0, kappa, [0])
    ref = oracle.ip_bruteforce(a, b, h, 0.0, 0, 20.0, kappa)
    assert np.array_equal(got[0], ref)
    assert abs(len(ref) / w - math.pi * r * r) < 0.01 * math.pi * r * r


def test_weight_one_is_the_single_photon_path():
    wl = synth.tiny_headon(n=2048, seed=44)
    a, b = synth.beams(wl)
    got, sp = gpu_ip_hits(a, b, 0.9, 0.3, wl.dt, wl.kappa, [0])
    ref, _ = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa)
    assert (got[0][:, 1] == 0).all() and (got[0][:, 3] == 0).all()
    assert np.array_equal(got[0][:, [0, 2]], ref)


def test_full_size_ip_workload_sampled_pairs():
    wl = synth.ip_headon()
    a, b = synth.beams(wl)
    h = synth.IP_CUBE_UM
    steps = [1, 2]
    got, sp = gpu_ip_hits(a, b, h, h, wl.dt, wl.kappa, steps)
    ma, mb = sp["mark_a"].cpu().numpy(), sp["mark_b"].cpu().numpy()
    assert sp["a"]["px"].numel() == int(a["w"][ma == 1].sum())
    rng = np.random.default_rng(45)
    sub = lambda beam, i: {k: v[i:i + 1].copy() for k, v in beam.items()}  # noqa: E731
    nb = len(mb)
    for k in steps:
        g = got[k]
        assert len(g) > 100000
        key = g[:, 0].astype(np.int64) * nb + g[:, 2]
        order = np.argsort(key, kind="stable")  # keeps (k, l) order inside a pair
        ks = key[order]
        uniq = np.unique(ks)
        pick = [int(x) for x in rng.choice(uniq, 150, replace=False)]
        # MP pairs with no real hit on the GPU, transversely near each other
        ia = rng.integers(0, len(ma), 4000)
        jb = rng.integers(0, nb, 4000)
        near_key = ia.astype(np.int64) * nb + jb
        close = ((np.abs(a["px"][ia] - b["px"][jb]) < 1.0) & (np.abs(a["py"][ia] - b["py"][jb]) < 1.0)
                 & ~np.isin(near_key, uniq))
        near = [int(x) for x in near_key[close][:150]]
        assert len(near) > 50
        for pk in pick + near:
            i, j = divmod(pk, nb)
            lo, hi = np.searchsorted(ks, pk, "left"), np.searchsorted(ks, pk, "right")
            mine = g[order[lo:hi]]
            ref = oracle.ip_bruteforce(sub(a, i), sub(b, j), h, h, k, wl.dt, wl.kappa).copy()
            ref[:, 0], ref[:, 2] = i, j
            assert np.array_equal(mine, ref), (k, i, j, len(mine), len(ref))


def test_edges():
    import torch
    wl, a, b = swarm_beams(50, 46, 3)
    A, B = binding.to_device(a), binding.to_device(b)
    # far apart: nothing can collide, nothing is written
    far = dict(B)
    far["px"] = B["px"] + 1000.0
    sp = binding.swarm_split(A, far, 0.5, 0.5, wl.dt, wl.kappa, 0, 1)
    assert sp["a"]["px"].numel() == 0 and sp["b"]["px"].numel() == 0
    assert int(sp["mark_a"].sum()) == 0
    # weights must be integers >= 1
    bad = dict(A)
    bad["w"] = A["w"].clone()
    bad["w"][7] = 1.5
    with pytest.raises(binding.TrilensError):
        binding.swarm_split(bad, B, 0.5, 0.5, wl.dt, wl.kappa, 0, 1)
    with pytest.raises(binding.TrilensError):
        binding.swarm_split(A, B, -0.5, 0.5, wl.dt, wl.kappa, 0, 1)
    torch.cuda.synchronize()
