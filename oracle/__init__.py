"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never calls it, and shares no code with it.

The C source (``oracle.c``) is compiled on first use with
``gcc -O2 -ffp-contract=off`` so that every FP64 operation is individually
rounded in the order written.  This module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source if missing or stale."""
    stale = (not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Beam(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [
        (k, ctypes.POINTER(ctypes.c_double)) for k in ("px", "py", "pz", "dx", "dy", "dz", "E", "w")
    ]


class Result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("weighted", ctypes.c_double),
                ("hsum", ctypes.c_uint64), ("hxor", ctypes.c_uint64),
                ("tests", ctypes.c_int64), ("node_tests", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d = ctypes.c_double
            L.oracle_ln.argtypes = [d]
            L.oracle_ln.restype = d
            L.oracle_sigma.argtypes = [d]
            L.oracle_sigma.restype = d
            L.oracle_s.argtypes = [d, d, d]
            L.oracle_s.restype = d
            L.oracle_sigma_max.argtypes = []
            L.oracle_sigma_max.restype = d
            L.oracle_splitmix64.argtypes = [ctypes.c_uint64]
            L.oracle_splitmix64.restype = ctypes.c_uint64
            pb = ctypes.POINTER(Beam)
            L.oracle_pair_hit.argtypes = [pb, ctypes.c_int64, pb, ctypes.c_int64, ctypes.c_int64, d, d]
            L.oracle_pair_hit.restype = ctypes.c_int
            L.oracle_pair_detail.argtypes = [pb, ctypes.c_int64, pb, ctypes.c_int64, ctypes.c_int64,
                                             d, d, ctypes.POINTER(ctypes.c_double)]
            L.oracle_pair_detail.restype = ctypes.c_int
            pu = ctypes.POINTER(ctypes.c_uint32)
            pr = ctypes.POINTER(Result)
            L.oracle_bruteforce.argtypes = [pb, pb, ctypes.c_int64, d, d, pu, ctypes.c_int64, pr]
            L.oracle_bruteforce.restype = ctypes.c_int
            L.oracle_tree.argtypes = [pb, pb, ctypes.c_int64, d, d, ctypes.c_int, ctypes.c_int, pu,
                                      ctypes.c_int64, pr]
            L.oracle_tree.restype = ctypes.c_int
            L.oracle_pair_products.argtypes = [pb, pb, pu, ctypes.c_int64, ctypes.c_uint64,
                                               ctypes.POINTER(ctypes.c_double)]
            L.oracle_pair_products.restype = ctypes.c_int
            L.oracle_com_direction.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.POINTER(ctypes.c_double)]
            L.oracle_com_direction.restype = None
            pd = ctypes.POINTER(ctypes.c_double)
            L.oracle_hit_times.argtypes = [pb, pb, ctypes.c_int64, d, d, pu, ctypes.c_int64, pd]
            L.oracle_hit_times.restype = ctypes.c_int
            L.oracle_deplete.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), pd, pu,
                                         pd, ctypes.c_int64, pd, ctypes.c_int64, pd]
            L.oracle_deplete.restype = ctypes.c_int
            L.oracle_swarm_offset.argtypes = [ctypes.c_uint64, pd]
            L.oracle_swarm_offset.restype = None
            L.oracle_ip_bruteforce.argtypes = [pb, pb, d, d, ctypes.c_int64, d, d, pu,
                                               ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
            L.oracle_ip_bruteforce.restype = ctypes.c_int
            pu32 = ctypes.POINTER(ctypes.c_uint32)
            L.oracle_cloud_pairs.argtypes = [pb, pb, ctypes.c_int64, d, d, pu32, ctypes.c_int64,
                                             pu32, ctypes.c_int64, pu32, ctypes.c_int64, pd, pd]
            L.oracle_cloud_pairs.restype = ctypes.c_int
            L.oracle_overlap_integral.argtypes = [pd] * 6 + [d]
            L.oracle_overlap_integral.restype = d
            _lib = L
    return _lib


def ln(x: float) -> float:
    return lib().oracle_ln(float(x))


def sigma(s: float) -> float:
    """Eq. BWcross [m^2]."""
    return lib().oracle_sigma(float(s))


def s_invariant(E1: float, E2: float, cos_phi: float) -> float:
    return lib().oracle_s(float(E1), float(E2), float(cos_phi))


def sigma_max() -> float:
    return lib().oracle_sigma_max()


def splitmix64(x: int) -> int:
    return lib().oracle_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF))


_KEYS = ("px", "py", "pz", "dx", "dy", "dz", "E", "w")


def _beam(b: dict) -> tuple[Beam, list]:
    keep = [np.ascontiguousarray(b[k], dtype=np.float64) for k in _KEYS]
    n = len(keep[0])
    for a in keep:
        assert a.shape == (n,)
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in keep]
    return Beam(n, *ptrs), keep


def pair_detail(a: dict, i: int, b: dict, j: int, step: int, dt: float, kappa: float):
    """(hit, s, sigma, r2, tstar, d2, vv) for one pair."""
    A, ka = _beam(a)
    B, kb = _beam(b)
    out = (ctypes.c_double * 6)()
    hit = lib().oracle_pair_detail(ctypes.byref(A), i, ctypes.byref(B), j, step, dt, kappa, out)
    return (bool(hit),) + tuple(out)


def _run(fn, a, b, step, dt, kappa, extra, cap):
    A, ka = _beam(a)
    B, kb = _beam(b)
    res = Result()
    for _ in range(3):
        hits = np.zeros((max(cap, 1), 2), dtype=np.uint32)
        rc = fn(ctypes.byref(A), ctypes.byref(B), int(step), float(dt), float(kappa), *extra,
                hits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap, ctypes.byref(res))
        if rc != 0:
            raise RuntimeError(f"oracle failed rc={rc}")
        if res.count <= cap:
            return hits[: res.count].copy(), res.as_dict()
        cap = int(res.count)
    raise RuntimeError("oracle capacity loop")


def bruteforce(a: dict, b: dict, step: int, dt: float, kappa: float, cap: int = 1 << 16):
    """All N_A x N_B pairs.  Returns (hits[n,2] uint32 lexicographic, result dict)."""
    return _run(lib().oracle_bruteforce, a, b, step, dt, kappa, (), cap)


def tree(a: dict, b: dict, step: int, dt: float, kappa: float, leaf_size: int = 8,
         nthreads: int = 1, cap: int = 1 << 16):
    """The paper's k-d hierarchy with depth-first dual traversal; same output."""
    return _run(lib().oracle_tree, a, b, step, dt, kappa, (int(leaf_size), int(nthreads)), cap)


def pair_products(a: dict, b: dict, hits, seed: int):
    """Electron and positron four-momenta [MeV] of each hit (i, j): (n, 8) float64
    = electron (E, px, py, pz), positron (E, px, py, pz)."""
    A, ka = _beam(a)
    B, kb = _beam(b)
    h = np.ascontiguousarray(np.asarray(hits, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros((len(h), 8), dtype=np.float64)
    rc = lib().oracle_pair_products(ctypes.byref(A), ctypes.byref(B),
                                    h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), len(h),
                                    ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("a hit's photon pair is below threshold")
    return out


def com_direction(seed: int, i: int, j: int) -> np.ndarray:
    """The CoM direction drawn for hit (i, j)."""
    n = (ctypes.c_double * 3)()
    lib().oracle_com_direction(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), i, j, n)
    return np.array(list(n))


def _pd(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def hit_times(a: dict, b: dict, step: int, dt: float, kappa: float, hits) -> np.ndarray:
    """Closest-approach time t* [fs, relative to t_k] of each hit (i, j) of step k."""
    A, ka = _beam(a)
    B, kb = _beam(b)
    h = np.ascontiguousarray(np.asarray(hits, dtype=np.uint32).reshape(-1, 2))
    t = np.zeros(len(h), dtype=np.float64)
    rc = lib().oracle_hit_times(ctypes.byref(A), ctypes.byref(B), int(step), float(dt),
                                float(kappa), h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                len(h), _pd(t))
    if rc != 0:
        raise ValueError("a listed pair is not a hit of this step")
    return t


def deplete(steps, tstar, hits, rem_a, rem_b):
    """Depletion in chronological order (Sec. 2.2, Sec. 3.1): the hits, each with its
    step and t*, taken in (step, t*, i, j) order; each takes min(rem_i, rem_j) from both.
    Returns (delta per hit, rem_a, rem_b after), leaving the inputs untouched."""
    h = np.ascontiguousarray(np.asarray(hits, dtype=np.uint32).reshape(-1, 2))
    n = len(h)
    st = np.ascontiguousarray(np.broadcast_to(np.asarray(steps, dtype=np.int64), (n,)))
    t = np.ascontiguousarray(np.asarray(tstar, dtype=np.float64).reshape(n))
    ra = np.array(rem_a, dtype=np.float64, copy=True)
    rb = np.array(rem_b, dtype=np.float64, copy=True)
    delta = np.zeros(n, dtype=np.float64)
    rc = lib().oracle_deplete(n, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _pd(t),
                              h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _pd(ra), len(ra),
                              _pd(rb), len(rb), _pd(delta))
    if rc == -1:
        raise ValueError("hit index out of range")
    if rc != 0:
        raise MemoryError("oracle_deplete")
    return delta, ra, rb


def deplete_run(a: dict, b: dict, dt: float, kappa: float, steps, rem_a=None, rem_b=None,
                use_tree: bool = True):
    """The exact hits of each step (in order), then depletion in time order across
    the steps.  Returns a list of (hits, delta) per step and the final (rem_a, rem_b);
    rem defaults to the weights."""
    ra = np.array(a["w"] if rem_a is None else rem_a, dtype=np.float64, copy=True)
    rb = np.array(b["w"] if rem_b is None else rem_b, dtype=np.float64, copy=True)
    out = []
    for k in steps:
        hits, _ = (tree if use_tree else bruteforce)(a, b, k, dt, kappa)
        t = hit_times(a, b, k, dt, kappa, hits)
        delta, ra, rb = deplete(k, t, hits, ra, rb)
        out.append((hits, delta))
    return out, ra, rb


def swarm_offset(k: int) -> np.ndarray:
    """Offset u_k (in units of the MP's cube side) of photon k of a swarm (IP regime)."""
    u = np.zeros(3)
    lib().oracle_swarm_offset(ctypes.c_uint64(k), _pd(u))
    return u


def ip_bruteforce(a: dict, b: dict, h_a: float, h_b: float, step: int, dt: float,
                  kappa: float, cap: int = 1 << 16):
    """IP regime (Sec. 2.2): every real-photon pair of the two beams' swarms.
    Returns hits[n, 4] uint32 = (MP i of a, photon k, MP j of b, photon l), sorted."""
    A, ka = _beam(a)
    B, kb = _beam(b)
    count = ctypes.c_int64(0)
    for _ in range(3):
        hits = np.zeros((max(cap, 1), 4), dtype=np.uint32)
        rc = lib().oracle_ip_bruteforce(ctypes.byref(A), ctypes.byref(B), float(h_a),
                                        float(h_b), int(step), float(dt), float(kappa),
                                        hits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                        cap, ctypes.byref(count))
        if rc == -1:
            raise ValueError("IP regime: weights must be integers in [1, 2^32)")
        if rc != 0:
            raise MemoryError("oracle_ip_bruteforce")
        if count.value <= cap:
            return hits[: count.value].copy()
        cap = int(count.value)
    raise RuntimeError("oracle capacity loop")


def _pu32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def cloud_pairs(a: dict, b: dict, step: int, dt: float, kappa: float, cloud_a, cloud_b, pairs):
    """Statistical regime at a cut (Sec. 2.2, Eq. rate, Eq. reactivity): clouds
    are given by photon -> cloud memberships; for every listed cloud pair
    (cloud of a, cloud of b) the 24 node-pair features and the ST rate (the
    expected number of pairs in step k).  Returns (feat[m, 24], st[m])."""
    A, ka = _beam(a)
    B, kb = _beam(b)
    ca = np.ascontiguousarray(cloud_a, dtype=np.uint32)
    cb = np.ascontiguousarray(cloud_b, dtype=np.uint32)
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.uint32).reshape(-1, 2))
    m = len(pr)
    assert len(ca) == len(a["px"]) and len(cb) == len(b["px"])
    nca = int(ca.max()) + 1 if len(ca) else 0
    ncb = int(cb.max()) + 1 if len(cb) else 0
    feat = np.zeros((m, 24))
    st = np.zeros(m)
    rc = lib().oracle_cloud_pairs(ctypes.byref(A), ctypes.byref(B), int(step), float(dt),
                                  float(kappa), _pu32(ca), nca, _pu32(cb), ncb, _pu32(pr), m,
                                  _pd(feat), _pd(st))
    if rc == -1:
        raise ValueError("cloud membership or pair out of range, or an empty cloud")
    if rc != 0:
        raise MemoryError("oracle_cloud_pairs")
    return feat, st


def overlap_integral(la, ua, va, lb, ub, vb, T: float) -> float:
    """Exact integral over [0, T] of the overlap volume of two moving boxes."""
    arr = [np.ascontiguousarray(x, dtype=np.float64) for x in (la, ua, va, lb, ub, vb)]
    return lib().oracle_overlap_integral(*[_pd(x) for x in arr], float(T))


def cloud_labels(a: dict, b: dict, hits, cloud_a, cloud_b, pairs):
    """Exact yield of every listed cloud pair: the sum of w_i w_j over the
    hits (i, j) whose photons lie in the pair's clouds, added in hit order.
    Returns (label[m], hits that fall in no listed pair)."""
    h = np.asarray(hits, dtype=np.int64).reshape(-1, 2)
    pr = np.asarray(pairs, dtype=np.uint64).reshape(-1, 2)
    ca = np.asarray(cloud_a, dtype=np.uint64)
    cb = np.asarray(cloud_b, dtype=np.uint64)
    key = (ca[h[:, 0]] << np.uint64(32)) | cb[h[:, 1]]
    pk = (pr[:, 0] << np.uint64(32)) | pr[:, 1]
    order = np.argsort(pk, kind="stable")
    spk = pk[order]
    pos = np.searchsorted(spk, key)
    pos_c = np.minimum(pos, max(len(spk) - 1, 0))
    found = (pos < len(spk)) & (spk[pos_c] == key) if len(spk) else np.zeros(len(key), bool)
    wa = np.asarray(a["w"], dtype=np.float64)
    wb = np.asarray(b["w"], dtype=np.float64)
    label = np.zeros(len(pr))
    np.add.at(label, order[pos_c[found]], wa[h[found, 0]] * wb[h[found, 1]])
    return label, int((~found).sum())
