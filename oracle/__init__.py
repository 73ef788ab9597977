"""FP64 CPU oracle of the deep potential -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2602_02234_b300``) and never imports it; the two meet only in the
seeded generators of ``synth``.

The arithmetic is plain C (``af_oracle.c``, ``afmp_oracle.c``, ``gf_oracle.c``)
in double precision; this file only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


_D, _I = C.c_double, C.c_int32
_PD, _PI = C.POINTER(C.c_double), C.POINTER(C.c_int32)


def _declare(L):
    L.oracle_af_weight_count.restype = C.c_longlong
    L.oracle_af_weight_count.argtypes = [_PI, _PD]
    L.oracle_af_weight_offset.restype = C.c_longlong
    L.oracle_af_weight_offset.argtypes = [_PI, _PD, C.c_int, C.c_int]
    L.oracle_neighbours.restype = C.c_int
    L.oracle_neighbours.argtypes = [C.c_int, _PD, _PD, C.c_double, C.c_int, C.c_int, _PI,
                                    C.c_int, _PI, _PI, _PI, _PD]
    L.oracle_af_atoms.restype = C.c_int
    L.oracle_af_atoms.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, C.c_int, _PI, C.c_int,
                                  _PD, _PD, _PI, _PI, _PD]
    L.oracle_af_compute.restype = C.c_int
    L.oracle_af_compute.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, C.c_int, _PD, _PD,
                                    _PD, _PD]
    L.oracle_af_md.restype = C.c_int
    L.oracle_af_md.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, _PD, _PD, C.c_int,
                               C.c_double, C.c_int, _PD, _PD]
    L.oracle_afmp_weight_count.restype = C.c_longlong
    L.oracle_afmp_weight_count.argtypes = [_PI, _PD]
    L.oracle_afmp_weight_offset.restype = C.c_longlong
    L.oracle_afmp_weight_offset.argtypes = [_PI, _PD, C.c_int, C.c_int]
    L.oracle_afmp_compute.restype = C.c_int
    L.oracle_afmp_compute.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, C.c_int, _PD, _PD,
                                      _PD, _PD]
    L.oracle_afmp_compute_seeded.restype = C.c_int
    L.oracle_afmp_compute_seeded.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, C.c_int, _PD,
                                             _PD, _PD, _PD, _PD]
    L.oracle_gf_compute_seeded.restype = C.c_int
    L.oracle_gf_compute_seeded.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, C.c_int, _PD,
                                           _PD, _PD, _PD, _PD]
    L.oracle_switch.restype = None
    L.oracle_switch.argtypes = [C.c_double, C.c_double, C.c_double, _PD, _PD]
    if hasattr(L, "oracle_gf_compute"):
        L.oracle_gf_weight_count.restype = C.c_longlong
        L.oracle_gf_weight_count.argtypes = [_PI, _PD]
        L.oracle_gf_weight_offset.restype = C.c_longlong
        L.oracle_gf_weight_offset.argtypes = [_PI, _PD, C.c_int, C.c_int]
        L.oracle_gf_compute.restype = C.c_int
        L.oracle_gf_compute.argtypes = [_PI, _PD, _PD, C.c_int, _PI, _PD, _PD, C.c_int, _PD,
                                        _PD, _PD, _PD]


# --------------------------------------------------------------------------
# model description marshalling
# --------------------------------------------------------------------------
def _af_dims(model):
    d = model if isinstance(model, dict) else model.as_dict()
    idims = np.array([d["n_species"], d["e1"], d["e2"], d["m1"], d["m2"], d["n_layers"],
                      d["hidden"], d["heads"], d["f1"], d["f2"], d["f3"], d["nmax"]], dtype=np.int32)
    fdims = np.array([d["rc"], d["rs"]], dtype=np.float64)
    return idims, fdims


def _gf_dims(model):
    d = model if isinstance(model, dict) else model.as_dict()
    idims = np.array([d["n_species"], d["node"], d["edge"], d["n_layers"], d["f1"], d["f2"],
                      d["f3"], d["nmax"], d["na"]], dtype=np.int32)
    fdims = np.array([d["rc"], d["rs"], d["rca"], d["rsa"]], dtype=np.float64)
    return idims, fdims


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


AF_KINDS = {"eW1": 0, "eb1": 1, "eW2": 2, "eb2": 3, "eW3": 4, "eb3": 5,
            "Wq": 10, "Wk": 11, "Wv": 12, "Wo": 13, "bo": 14,
            "fW1": 20, "fb1": 21, "fW2": 22, "fb2": 23, "fW3": 24, "fb3": 25, "fW4": 26, "fb4": 27}


def _mp(model) -> bool:
    d = model if isinstance(model, dict) else model.as_dict()
    return bool(d.get("message_passing", 0))


def af_weight_count(model) -> int:
    """Blob length; with k fitting heads the fitting nets of heads 1..k-1
    follow head 0's, in the same layout.  With message passing the blob also
    holds the atom-channel weights (afmp_oracle.c)."""
    i, f = _af_dims(model)
    if _mp(model):
        d = model if isinstance(model, dict) else model.as_dict()
        if max(1, d.get("fit_heads", 1)) != 1:
            raise ValueError("message passing takes one fitting head")
        n = lib().oracle_afmp_weight_count(_p(i, _I), _p(f, _D))
        if n < 0:
            raise ValueError("invalid attention-family model")
        return int(n)
    n = lib().oracle_af_weight_count(_p(i, _I), _p(f, _D))
    if n < 0:
        raise ValueError("invalid attention-family model")
    d = model if isinstance(model, dict) else model.as_dict()
    return int(n) + (max(1, d.get("fit_heads", 1)) - 1) * _af_fit_len(d)


def _af_fit_len(d):
    return d["n_species"] * (d["m1"] * d["m2"] * d["f1"] + d["f1"] + d["f1"] * d["f2"] + d["f2"]
                             + d["f2"] * d["f3"] + d["f3"] + d["f3"] + 1)


def af_head_blob(model, weights, h):
    """The single-head model of fitting head h: the shared embedding and
    attention weights followed by head h's fitting nets."""
    d = dict(model if isinstance(model, dict) else model.as_dict())
    d["fit_heads"] = 1
    n1 = af_weight_count(d)
    fl = _af_fit_len(d)
    w = np.asarray(weights, dtype=np.float64)
    shared = n1 - fl
    return np.concatenate([w[:shared], w[shared + h * fl: shared + (h + 1) * fl]]), d


def af_compute_heads(model, weights, types, coords, box, nthreads=0):
    """Multi-head fitting on one shared descriptor (paper Sec. II: a large
    atomic model with one fitting branch per training set), by definition: head
    h is the single-head model with head h's fitting nets.  Returns the energies
    of all heads and (E, atomic energies, forces, virial) of head 0."""
    d = model if isinstance(model, dict) else model.as_dict()
    k = max(1, d.get("fit_heads", 1))
    energies, head0 = [], None
    for h in range(k):
        wh, dh = af_head_blob(model, weights, h)
        r = af_compute(dh, wh, types, coords, box, nthreads)
        energies.append(r[0])
        if h == 0:
            head0 = r
    return np.array(energies), head0


def afmp_weight_slice(model, kind: str, a: int = 0) -> slice:
    """Message-passing blocks: ``Wt`` (species rows of the atom channel's
    initial value), ``Wm`` / ``bm`` of layer ``a``."""
    i, f = _af_dims(model)
    d = model if isinstance(model, dict) else model.as_dict()
    k = {"Wt": 0, "Wm": 1, "bm": 2}[kind]
    off = lib().oracle_afmp_weight_offset(_p(i, _I), _p(f, _D), k, a)
    if off < 0:
        raise ValueError((kind, a))
    size = {"Wt": d["n_species"] * d["m1"], "Wm": d["m1"] * d["m1"], "bm": d["m1"]}[kind]
    return slice(int(off), int(off) + size)


def af_weight_slice(model, kind: str, a: int) -> slice:
    """Slice of the blob holding block ``kind`` of species/layer ``a``."""
    if _mp(model):
        raise ValueError("use afmp_weight_slice for message-passing blobs")
    i, f = _af_dims(model)
    off = lib().oracle_af_weight_offset(_p(i, _I), _p(f, _D), AF_KINDS[kind], a)
    if off < 0:
        raise ValueError((kind, a))
    d = model if isinstance(model, dict) else model.as_dict()
    sizes = {"eW1": d["e1"], "eb1": d["e1"], "eW2": d["e1"] * d["e2"], "eb2": d["e2"],
             "eW3": d["e2"] * d["m1"], "eb3": d["m1"], "Wq": d["m1"] * d["hidden"],
             "Wk": d["m1"] * d["hidden"], "Wv": d["m1"] * d["hidden"], "Wo": d["hidden"] * d["m1"],
             "bo": d["m1"], "fW1": d["m1"] * d["m2"] * d["f1"], "fb1": d["f1"],
             "fW2": d["f1"] * d["f2"], "fb2": d["f2"], "fW3": d["f2"] * d["f3"], "fb3": d["f3"],
             "fW4": d["f3"], "fb4": 1}
    return slice(int(off), int(off) + sizes[kind])


def switch(r, rs, rc):
    """(sw, dsw/dr) of the smooth switch at distance r."""
    a, b = C.c_double(), C.c_double()
    lib().oracle_switch(float(r), float(rs), float(rc), C.byref(a), C.byref(b))
    return a.value, b.value


# --------------------------------------------------------------------------
# neighbours
# --------------------------------------------------------------------------
def neighbours(coords, box, rc, nmax, centres=None, use_cells=True):
    """Per centre: (count within rc, j[nmax], image[nmax,3], r[nmax,3]) in key order."""
    x = _c64(coords)
    n = len(x)
    cen = _c32(np.arange(n) if centres is None else centres)
    nc = len(cen)
    cnt = np.zeros(nc, np.int32)
    nj = np.zeros((nc, nmax), np.int32)
    ni = np.zeros((nc, nmax, 3), np.int32)
    nr = np.zeros((nc, nmax, 3), np.float64)
    b = _c64(box)
    rcode = lib().oracle_neighbours(n, _p(x, _D), _p(b, _D), float(rc), int(nmax), nc,
                                    _p(cen, _I), int(bool(use_cells)), _p(cnt, _I), _p(nj, _I),
                                    _p(ni, _I), _p(nr, _D))
    if rcode:
        raise RuntimeError("oracle_neighbours failed")
    return cnt, nj, ni, nr


# --------------------------------------------------------------------------
# attention family
# --------------------------------------------------------------------------
def af_compute(model, weights, types, coords, box, nthreads=0):
    """(E, atomic energies, forces N x 3, virial 3 x 3) in FP64."""
    i, f = _af_dims(model)
    w, t, x, b = _c64(weights), _c32(types), _c64(coords), _c64(box)
    if len(w) != af_weight_count(model):
        raise ValueError("weight blob has the wrong length")
    n = len(t)
    E = np.zeros(1)
    ae = np.zeros(n)
    F = np.zeros((n, 3))
    V = np.zeros((3, 3))
    fn = lib().oracle_afmp_compute if _mp(model) else lib().oracle_af_compute
    rc = fn(_p(i, _I), _p(f, _D), _p(w, _D), n, _p(t, _I), _p(x, _D),
                                 _p(b, _D), int(nthreads), _p(E, _D), _p(ae, _D), _p(F, _D),
                                 _p(V, _D))
    if rc:
        raise RuntimeError("attention-family oracle failed")
    return float(E[0]), ae, F, V


def compute_seeded(model, weights, types, coords, box, seed, nthreads=0):
    """E = sum_i seed_i e_i of a layer-coupled model (attention family with
    message passing, or graph family), its forces -dE/dx on every atom, the
    atomic energies e_i and the virial.  Atoms with seed 0 are ghosts: they
    take part as centres and neighbours, their own energy is not counted."""
    d = model if isinstance(model, dict) else model.as_dict()
    graph = "node" in d
    if not graph and not _mp(model):
        raise ValueError("seeded evaluation covers the layer-coupled models")
    i, f = _gf_dims(model) if graph else _af_dims(model)
    w, t, x, b = _c64(weights), _c32(types), _c64(coords), _c64(box)
    sd = _c64(seed)
    n = len(t)
    if len(sd) != n:
        raise ValueError("one seed per atom")
    E = np.zeros(1)
    ae = np.zeros(n)
    F = np.zeros((n, 3))
    V = np.zeros((3, 3))
    fn = lib().oracle_gf_compute_seeded if graph else lib().oracle_afmp_compute_seeded
    rc = fn(_p(i, _I), _p(f, _D), _p(w, _D), n, _p(t, _I), _p(x, _D), _p(b, _D), int(nthreads),
            _p(sd, _D), _p(E, _D), _p(ae, _D), _p(F, _D), _p(V, _D))
    if rc:
        raise RuntimeError("seeded oracle failed")
    return float(E[0]), ae, F, V


def af_compute_group(model, weights, types, coords, box, mask, nthreads=0):
    """The potential over a DP group (paper Sec. III: the deep potential covers
    a selected atom group): by definition the members evaluated alone in the
    same box, so only members see each other and carry energy; non-members get
    zero energy and force.  Returns (E, atomic energies, forces, virial)."""
    mask = np.asarray(mask, dtype=bool)
    idx = np.nonzero(mask)[0]
    n = len(mask)
    ae = np.zeros(n)
    F = np.zeros((n, 3))
    if len(idx) == 0:
        return 0.0, ae, F, np.zeros((3, 3))
    E, ae_g, F_g, V = af_compute(model, weights, np.asarray(types)[idx], np.asarray(coords)[idx],
                                 box, nthreads)
    ae[idx] = ae_g
    F[idx] = F_g
    return E, ae, F, V


def af_atoms(model, weights, types, coords, box, centres, nthreads=0, want_desc=False):
    """Per centre: atomic energy, pair gradients g (nmax x 3), neighbour j and image."""
    if _mp(model):
        raise ValueError("message passing couples every atom: use af_compute")
    i, f = _af_dims(model)
    d = model if isinstance(model, dict) else model.as_dict()
    nmax = d["nmax"]
    w, t, x, b = _c64(weights), _c32(types), _c64(coords), _c64(box)
    cen = _c32(centres)
    nc = len(cen)
    ae = np.zeros(nc)
    pg = np.zeros((nc, nmax, 3))
    pj = np.zeros((nc, nmax), np.int32)
    pim = np.zeros((nc, nmax, 3), np.int32)
    desc = np.zeros((nc, d["m1"] * d["m2"])) if want_desc else None
    rc = lib().oracle_af_atoms(_p(i, _I), _p(f, _D), _p(w, _D), len(t), _p(t, _I), _p(x, _D),
                               _p(b, _D), nc, _p(cen, _I), int(nthreads), _p(ae, _D), _p(pg, _D),
                               _p(pj, _I), _p(pim, _I), _p(desc, _D) if want_desc else None)
    if rc:
        raise RuntimeError("oracle_af_atoms failed")
    out = {"atom_e": ae, "pair_g": pg, "pair_j": pj, "pair_img": pim}
    if want_desc:
        out["desc"] = desc
    return out


def af_forces_subset(model, weights, types, coords, box, sample, nthreads=0):
    """Forces on the atoms in ``sample`` only (FP64), from the pair gradients of
    each sampled atom and of every atom that has a sampled atom as neighbour."""
    d = model if isinstance(model, dict) else model.as_dict()
    sample = np.asarray(sample, dtype=np.int32)
    # every centre whose (rc-)neighbourhood can contain a sampled atom
    cnt, nj, _, _ = neighbours(coords, box, d["rc"], 4096, centres=sample)
    need = set(int(s) for s in sample)
    for q in range(len(sample)):
        need.update(int(j) for j in nj[q, :cnt[q]])
    centres = np.array(sorted(need), dtype=np.int32)
    out = af_atoms(model, weights, types, coords, box, centres, nthreads)
    pos = {int(c): k for k, c in enumerate(centres)}
    F = np.zeros((len(sample), 3))
    for q, s in enumerate(sample):
        s = int(s)
        F[q] += out["pair_g"][pos[s]].sum(0)
    sidx = {int(s): q for q, s in enumerate(sample)}
    for k, c in enumerate(centres):
        for p in range(d["nmax"]):
            j = int(out["pair_j"][k, p])
            if j in sidx:
                F[sidx[j]] -= out["pair_g"][k, p]
    return F


def af_md(model, weights, types, masses, coords, vel, box, n_steps, dt, nthreads=0):
    """Velocity-Verlet NVE; returns (x, v, epot[n_steps], ekin[n_steps])."""
    if _mp(model):
        raise ValueError("af_md covers the model without message passing")
    i, f = _af_dims(model)
    w, t, m, b = _c64(weights), _c32(types), _c64(masses), _c64(box)
    x = _c64(coords).copy()
    v = _c64(vel).copy()
    ep = np.zeros(max(n_steps, 1))
    ek = np.zeros(max(n_steps, 1))
    rc = lib().oracle_af_md(_p(i, _I), _p(f, _D), _p(w, _D), len(t), _p(t, _I), _p(m, _D),
                            _p(b, _D), _p(x, _D), _p(v, _D), int(n_steps), float(dt),
                            int(nthreads), _p(ep, _D), _p(ek, _D))
    if rc:
        raise RuntimeError("oracle_af_md failed")
    return x, v, ep[:n_steps], ek[:n_steps]


# --------------------------------------------------------------------------
# graph family
# --------------------------------------------------------------------------
GF_KINDS = {"Wt": 0, "we": 1, "be0": 2, "Wm": 10, "Wn": 11, "bn": 12, "Wa": 13, "Wb": 14,
            "Wc": 15, "be": 16, "Wp": 17, "Wphi": 18, "Wq": 19, "bq": 20, "F1": 30, "c1": 31,
            "F2": 32, "c2": 33, "F3": 34, "c3": 35, "F4": 36, "c4": 37}


def gf_weight_count(model) -> int:
    i, f = _gf_dims(model)
    n = lib().oracle_gf_weight_count(_p(i, _I), _p(f, _D))
    if n < 0:
        raise ValueError("invalid graph-family model")
    return int(n)


def gf_weight_slice(model, kind: str, a: int = 0) -> slice:
    i, f = _gf_dims(model)
    off = lib().oracle_gf_weight_offset(_p(i, _I), _p(f, _D), GF_KINDS[kind], a)
    if off < 0:
        raise ValueError((kind, a))
    d = model if isinstance(model, dict) else model.as_dict()
    Nd, Ed = d["node"], d["edge"]
    sizes = {"Wt": d["n_species"] * Nd, "we": Ed, "be0": Ed, "Wm": Nd * Ed, "Wn": (Nd + Ed) * Nd,
             "bn": Nd, "Wa": Nd * Ed, "Wb": Nd * Ed, "Wc": Ed * Ed, "be": Ed, "Wp": Ed * Ed,
             "Wphi": 4 * Ed, "Wq": Ed * Ed, "bq": Ed, "F1": Nd * d["f1"], "c1": d["f1"],
             "F2": d["f1"] * d["f2"], "c2": d["f2"], "F3": d["f2"] * d["f3"], "c3": d["f3"],
             "F4": d["f3"], "c4": 1}
    return slice(int(off), int(off) + sizes[kind])


def gf_compute(model, weights, types, coords, box, nthreads=0):
    """(E, atomic energies, forces N x 3, virial 3 x 3) of the graph family, FP64."""
    i, f = _gf_dims(model)
    w, t, x, b = _c64(weights), _c32(types), _c64(coords), _c64(box)
    if len(w) != gf_weight_count(model):
        raise ValueError("weight blob has the wrong length")
    n = len(t)
    E = np.zeros(1)
    ae = np.zeros(n)
    F = np.zeros((n, 3))
    V = np.zeros((3, 3))
    rc = lib().oracle_gf_compute(_p(i, _I), _p(f, _D), _p(w, _D), n, _p(t, _I), _p(x, _D),
                                 _p(b, _D), int(nthreads), _p(E, _D), _p(ae, _D), _p(F, _D),
                                 _p(V, _D))
    if rc:
        raise RuntimeError("oracle_gf_compute failed")
    return float(E[0]), ae, F, V


KAPPA = 1.602176634e-19 / (1.66053906660e-27 * 1e10)
