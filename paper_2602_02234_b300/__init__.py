"""Python binding of libdp.so: deep-potential energy/force inference and MD on one B300.

Argument marshalling only -- every step of the computation runs in the CUDA
kernels of ``libdp.so`` (built for sm_103a by ``paper_2602_02234_b300.build``).
There is no CPU or PyTorch fallback: importing the binding without the built
library raises, and so does any call that the library rejects.

The names follow the C ABI of ``include/dp.h``:

* ``ModelDesc``  -- ``dp_model_desc``
* ``weight_count`` -- ``dp_weight_count``
* ``DeepPotential`` -- a ``dp_ctx``: ``compute`` (``dp_compute``), ``step``
  (``dp_step``), ``get_state``/``set_state``, ``neighbours``,
  ``atom_energies``, ``head_energies`` (``dp_get_head_energies``),
  ``set_group`` (``dp_set_group``), ``set_centres`` (``dp_set_centres``),
  ``set_energy_seed`` (``dp_set_energy_seed``),
  ``kernels_per_step``, ``device_bytes``
* ``Server`` -- ``dp_server_*``: continuous batching of independent systems
* ``DPEnergy`` -- ``torch.autograd.Function`` whose forward is ``dp_compute``
  and whose backward returns -dE/dx * grad (forces from the hand-written
  adjoint kernels).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdp.so")

DP_OK, DP_ERR_ARG, DP_ERR_OOM, DP_ERR_NLIST_OVERFLOW, DP_ERR_TIMEOUT = 0, -1, -2, -3, -4
DP_ERR_NONFINITE, DP_ERR_CUDA, DP_ERR_UNSUPPORTED = -5, -6, -7
FAMILY_ATTENTION, FAMILY_GRAPH = 0, 1
PREC_PLAIN_F64, PREC_PLAIN_F32, PREC_FUSED = 0, 1, 2
PTR_HOST, PTR_DEVICE = 0, 1

_ERRNAMES = {DP_ERR_ARG: "DP_ERR_ARG", DP_ERR_OOM: "DP_ERR_OOM",
             DP_ERR_NLIST_OVERFLOW: "DP_ERR_NLIST_OVERFLOW", DP_ERR_TIMEOUT: "DP_ERR_TIMEOUT",
             DP_ERR_NONFINITE: "DP_ERR_NONFINITE", DP_ERR_CUDA: "DP_ERR_CUDA",
             DP_ERR_UNSUPPORTED: "DP_ERR_UNSUPPORTED"}


class DPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class ModelDesc(C.Structure):
    _fields_ = [("family", C.c_int), ("precision", C.c_int), ("n_species", C.c_int),
                ("nmax", C.c_int), ("rcut", C.c_double), ("rcut_smth", C.c_double),
                ("e1", C.c_int), ("e2", C.c_int), ("m1", C.c_int), ("m2", C.c_int),
                ("n_layers", C.c_int), ("hidden", C.c_int), ("heads", C.c_int),
                ("node_dim", C.c_int), ("edge_dim", C.c_int), ("n_gnn_layers", C.c_int),
                ("angle_nmax", C.c_int), ("angle_rcut", C.c_double),
                ("angle_rcut_smth", C.c_double), ("f1", C.c_int), ("f2", C.c_int),
                ("f3", C.c_int), ("skin", C.c_double), ("rebuild_every", C.c_int),
                ("fit_heads", C.c_int), ("message_passing", C.c_int),
                ("reserved", C.c_int * 5)]


def model_desc(model, precision: int, skin: float = 1.0, rebuild_every: int = 10) -> ModelDesc:
    """A ``dp_model_desc`` from a dict (or object with ``as_dict``) of model sizes.

    Attention family keys: n_species e1 e2 m1 m2 n_layers hidden heads f1 f2 f3
    nmax rc rs, and optionally fit_heads (fitting heads on one descriptor) and
    message_passing (0/1: the atom channel passed between neighbours every
    layer).  Graph family keys: n_species node edge n_layers f1 f2 f3 nmax na
    rc rs rca rsa.  precision: PREC_PLAIN_F64, PREC_PLAIN_F32 or PREC_FUSED
    (16-bit tensor-core operands; for the graph family the mixed form).
    """
    d = model if isinstance(model, dict) else model.as_dict()
    m = ModelDesc()
    m.precision = precision
    m.n_species = d["n_species"]
    m.nmax = d["nmax"]
    m.rcut = d["rc"]
    m.rcut_smth = d["rs"]
    m.f1, m.f2, m.f3 = d["f1"], d["f2"], d["f3"]
    m.skin = skin
    m.rebuild_every = rebuild_every
    if "node" in d:
        m.family = FAMILY_GRAPH
        m.node_dim, m.edge_dim, m.n_gnn_layers = d["node"], d["edge"], d["n_layers"]
        m.angle_nmax, m.angle_rcut, m.angle_rcut_smth = d["na"], d["rca"], d["rsa"]
    else:
        m.family = FAMILY_ATTENTION
        m.e1, m.e2, m.m1, m.m2 = d["e1"], d["e2"], d["m1"], d["m2"]
        m.n_layers, m.hidden, m.heads = d["n_layers"], d["hidden"], d["heads"]
        m.fit_heads = d.get("fit_heads", 1)
        m.message_passing = d.get("message_passing", 0)
    return m


_lib = None


def lib():
    """The loaded libdp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdp.so is not built ({LIB_PATH}); run "
                              "`python -m paper_2602_02234_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.dp_weight_count.argtypes = [C.POINTER(ModelDesc), C.POINTER(C.c_size_t)]
        L.dp_init.argtypes = [C.POINTER(vp), C.POINTER(ModelDesc), i, vp, vp, vp, vp, C.c_size_t, vp]
        L.dp_compute.argtypes = [vp, vp, vp, vp, vp, i]
        L.dp_step.argtypes = [vp, i, d, vp, vp, vp, i]
        L.dp_get_state.argtypes = [vp, vp, vp, C.POINTER(C.c_longlong), i]
        L.dp_set_state.argtypes = [vp, vp, vp, C.c_longlong, i]
        L.dp_get_neighbours.argtypes = [vp, vp, vp, vp]
        L.dp_get_atom_energies.argtypes = [vp, vp]
        L.dp_set_group.argtypes = [vp, vp]
        L.dp_set_centres.argtypes = [vp, vp]
        L.dp_set_energy_seed.argtypes = [vp, vp]
        L.dp_get_head_energies.argtypes = [vp, vp]
        L.dp_enqueue_network.argtypes = [vp, i, i]
        L.dp_kernels_per_step.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.dp_device_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.dp_neighbour_list_noalloc.argtypes = [vp, i, vp, d, i, vp, vp, vp, vp]
        L.dp_noalloc_last_error.argtypes = []
        L.dp_noalloc_last_error.restype = C.c_char_p
        L.dp_selftest_mma.argtypes = [i, i, i, i, i, vp, vp, vp]
        L.dp_selftest_timeout.argtypes = [C.c_longlong]
        L.dp_selftest_mma_rate.argtypes = [i, i, i, C.POINTER(C.c_double)]
        L.dp_server_create.argtypes = [C.POINTER(vp), C.POINTER(ModelDesc), vp, vp, C.c_size_t, i,
                                       C.c_longlong, C.c_size_t, d, vp]
        L.dp_server_capacity.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.dp_server_submit.argtypes = [vp, i, vp, vp, vp, vp, i, C.POINTER(C.c_uint64)]
        L.dp_server_tick.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.dp_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int), vp, vp, vp, vp]
        L.dp_server_stats.argtypes = [vp, vp, i]
        L.dp_server_free.argtypes = [vp]
        L.dp_server_free.restype = None
        L.dp_server_last_error.argtypes = [vp]
        L.dp_server_last_error.restype = C.c_char_p
        L.dp_free.argtypes = [vp]
        L.dp_free.restype = None
        L.dp_last_error.argtypes = [vp]
        L.dp_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def weight_count(desc: ModelDesc) -> int:
    n = C.c_size_t()
    rc = lib().dp_weight_count(C.byref(desc), C.byref(n))
    if rc:
        raise DPError(rc, lib().dp_last_error(None).decode())
    return int(n.value)


def _ptr(a):
    """(address, kind) of a numpy array or a torch tensor."""
    if a is None:
        return None, PTR_HOST
    if isinstance(a, np.ndarray):
        return a.ctypes.data, PTR_HOST
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.data_ptr(), (PTR_DEVICE if a.is_cuda else PTR_HOST)
    except ImportError:  # pragma: no cover
        pass
    raise TypeError(type(a))


class DeepPotential:
    """One system (``dp_ctx``): species, box and weights are fixed at creation."""

    def __init__(self, desc: ModelDesc, types, box, weights, masses=None, stream=None):
        self.desc = desc
        self.types = np.ascontiguousarray(types, dtype=np.int32)
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        self.n = len(self.types)
        m = None if masses is None else np.ascontiguousarray(masses, dtype=np.float64)
        h = C.c_void_p()
        st = None
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = lib().dp_init(C.byref(h), C.byref(desc), self.n, self.types.ctypes.data,
                           None if m is None else m.ctypes.data, self.box.ctypes.data,
                           w.ctypes.data, len(w), st)
        if rc:
            raise DPError(rc, lib().dp_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc:
            raise DPError(rc, lib().dp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().dp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- compute
    def compute(self, coords, forces=None, virial=None):
        """E (float) and, into the given buffers, forces (N x 3) and virial (3 x 3).

        numpy arguments are host memory; CUDA tensors are device memory (all
        arguments of one call must be of the same kind).  Returns (E, F, V).
        """
        xp, kind = _ptr(coords)
        if kind == PTR_HOST:
            coords = np.ascontiguousarray(coords, dtype=np.float64)
            xp = coords.ctypes.data
            if forces is None:
                forces = np.zeros((self.n, 3))
            if virial is None:
                virial = np.zeros((3, 3))
            e = np.zeros(1)
            self._check(lib().dp_compute(self._h, xp, e.ctypes.data, forces.ctypes.data,
                                         virial.ctypes.data, PTR_HOST))
            return float(e[0]), forces, virial
        import torch
        dev = coords.device
        if forces is None:
            forces = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        if virial is None:
            virial = torch.empty((3, 3), dtype=torch.float64, device=dev)
        e = torch.empty(1, dtype=torch.float64, device=dev)
        self._check(lib().dp_compute(self._h, xp, e.data_ptr(), forces.data_ptr(),
                                     virial.data_ptr(), PTR_DEVICE))
        return e, forces, virial

    def step(self, n_steps, dt_fs, coords=None, vel=None, energies=False):
        """``n_steps`` of velocity Verlet.  coords/vel (numpy, updated in place)
        are uploaded first when given; otherwise the resident state is used.
        Returns the per-step (E_pot, E_kin) array when ``energies``."""
        tr = np.zeros((max(n_steps, 1), 2)) if energies else None
        if coords is not None:
            assert coords.dtype == np.float64 and coords.flags["C_CONTIGUOUS"]
        if vel is not None:
            assert vel.dtype == np.float64 and vel.flags["C_CONTIGUOUS"]
        self._check(lib().dp_step(self._h, int(n_steps), float(dt_fs),
                                  None if coords is None else coords.ctypes.data,
                                  None if vel is None else vel.ctypes.data,
                                  None if tr is None else tr.ctypes.data, PTR_HOST))
        return tr[:n_steps] if energies else None

    def get_state(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        s = C.c_longlong()
        self._check(lib().dp_get_state(self._h, x.ctypes.data, v.ctypes.data, C.byref(s), PTR_HOST))
        return x, v, int(s.value)

    def set_state(self, coords, vel, step=0):
        x = np.ascontiguousarray(coords, dtype=np.float64)
        v = np.ascontiguousarray(vel, dtype=np.float64)
        self._check(lib().dp_set_state(self._h, x.ctypes.data, v.ctypes.data, int(step), PTR_HOST))

    # --------------------------------------------------------------- inspection
    def neighbours(self):
        nm = self.desc.nmax
        j = np.zeros((self.n, nm), np.int32)
        img = np.zeros((self.n, nm, 3), np.int32)
        cnt = np.zeros(self.n, np.int32)
        self._check(lib().dp_get_neighbours(self._h, j.ctypes.data, img.ctypes.data, cnt.ctypes.data))
        return cnt, j, img

    def head_energies(self):
        """Energy of every fitting head at the last evaluation (head 0 first;
        dp_get_head_energies)."""
        k = max(1, self.desc.fit_heads) if self.desc.family == FAMILY_ATTENTION else 1
        e = np.zeros(k)
        self._check(lib().dp_get_head_energies(self._h, e.ctypes.data))
        return e

    def set_group(self, mask=None):
        """DP group: a boolean array over the atoms (None: every atom).  Only
        pairs of members interact through the potential; non-members get zero
        energy and force (dp_set_group)."""
        if mask is None:
            self._check(lib().dp_set_group(self._h, None))
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=bool), dtype=np.uint8)
        if m.shape != (self.n,):
            raise ValueError("mask must have one entry per atom")
        self._check(lib().dp_set_group(self._h, m.ctypes.data))

    def set_centres(self, mask=None):
        """Centres of a domain-decomposed subdomain: a boolean array over the
        local atoms (owned True, ghosts False; None: every atom).  Only centres
        carry energy; forces are the centres' partial forces on every local
        atom (dp_set_centres)."""
        if mask is None:
            self._check(lib().dp_set_centres(self._h, None))
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=bool), dtype=np.uint8)
        if m.shape != (self.n,):
            raise ValueError("mask must have one entry per atom")
        self._check(lib().dp_set_centres(self._h, m.ctypes.data))

    def set_energy_seed(self, mask=None):
        """Energy seed of a subdomain (any model; needed by layer-coupled ones):
        a boolean array over the local atoms (owned True).  Every atom is a
        centre, only owned energies count and seed the adjoint
        (dp_set_energy_seed)."""
        if mask is None:
            self._check(lib().dp_set_energy_seed(self._h, None))
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=bool), dtype=np.uint8)
        if m.shape != (self.n,):
            raise ValueError("mask must have one entry per atom")
        self._check(lib().dp_set_energy_seed(self._h, m.ctypes.data))

    def atom_energies(self):
        e = np.zeros(self.n)
        self._check(lib().dp_get_atom_energies(self._h, e.ctypes.data))
        return e

    def enqueue_network(self, reps=1, parts=0):
        """Enqueue the network kernels alone ``reps`` times (no sync); ``parts``
        selects kernels (0 = all; fused: 1 forward, 2 fitting, 4 backward)."""
        self._check(lib().dp_enqueue_network(self._h, int(reps), int(parts)))

    def kernels_per_step(self):
        a, b = C.c_int(), C.c_int()
        self._check(lib().dp_kernels_per_step(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def device_bytes(self):
        b = C.c_size_t()
        self._check(lib().dp_device_bytes(self._h, C.byref(b)))
        return int(b.value)


class Server:
    """``dp_server``: continuous batching of independent systems (fused model)."""

    STATS = ("ticks", "p50_tick_ms", "p99_tick_ms", "atom_steps", "busy_ms", "max_resident",
             "max_resident_atoms", "waits_for_memory", "waits_for_slot", "atom_capacity")

    def __init__(self, desc, weights, masses, max_slots=64, max_atoms=0, mem_budget=0,
                 dt_fs=0.5, stream=None):
        w = np.ascontiguousarray(weights, dtype=np.float64)
        m = np.ascontiguousarray(masses, dtype=np.float64)
        h = C.c_void_p()
        st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = lib().dp_server_create(C.byref(h), C.byref(desc), m.ctypes.data, w.ctypes.data, len(w),
                                    int(max_slots), int(max_atoms), int(mem_budget), float(dt_fs), st)
        if rc:
            raise DPError(rc, lib().dp_server_last_error(None).decode())
        self._h = h
        self.sizes = {}

    def _check(self, rc):
        if rc:
            raise DPError(rc, lib().dp_server_last_error(self._h).decode())

    def capacity(self):
        a, s = C.c_int(), C.c_int()
        self._check(lib().dp_server_capacity(self._h, C.byref(a), C.byref(s)))
        return a.value, s.value

    def submit(self, types, box, coords, vel, n_steps):
        t = np.ascontiguousarray(types, dtype=np.int32)
        b = np.ascontiguousarray(box, dtype=np.float64)
        x = np.ascontiguousarray(coords, dtype=np.float64)
        v = np.ascontiguousarray(vel, dtype=np.float64)
        rid = C.c_uint64()
        self._check(lib().dp_server_submit(self._h, len(t), t.ctypes.data, b.ctypes.data,
                                           x.ctypes.data, v.ctypes.data, int(n_steps), C.byref(rid)))
        self.sizes[rid.value] = (len(t), int(n_steps))
        return rid.value

    def tick(self):
        a, q = C.c_int(), C.c_int()
        self._check(lib().dp_server_tick(self._h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def poll(self, rid):
        """None while queued or running; else (coords, vel, energies, latency)."""
        n, steps = self.sizes[rid]
        st = C.c_int()
        x = np.zeros((n, 3))
        v = np.zeros((n, 3))
        e = np.zeros((steps, 2))
        lat = np.zeros(4)
        self._check(lib().dp_server_poll(self._h, C.c_uint64(rid), C.byref(st), x.ctypes.data,
                                         v.ctypes.data, e.ctypes.data, lat.ctypes.data))
        if st.value != 2:
            return None
        return x, v, e, {"total_ms": lat[0], "queue_ms": lat[1], "tick_admitted": int(lat[2]),
                         "tick_done": int(lat[3])}

    def stats(self):
        out = np.zeros(len(self.STATS))
        self._check(lib().dp_server_stats(self._h, out.ctypes.data, len(out)))
        return dict(zip(self.STATS, out.tolist()))

    def close(self):
        if getattr(self, "_h", None):
            lib().dp_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def neighbour_list_noalloc(coords, box, rcut, nmax, stream=None):
    """``dp_neighbour_list_noalloc``: neighbour lists of one small system
    (<= 1024 atoms) with no device allocation by the library.  ``coords`` is a
    CUDA float64 tensor (N x 3); the output tensors are allocated here by torch
    (the caller's side).  Returns (n_in_rc, nbr_j, nbr_img) as CUDA tensors."""
    import torch
    assert coords.is_cuda and coords.dtype == torch.float64 and coords.is_contiguous()
    n = coords.shape[0]
    dev = coords.device
    j = torch.empty((n, nmax), dtype=torch.int32, device=dev)
    img = torch.empty((n, nmax, 3), dtype=torch.int32, device=dev)
    cnt = torch.empty((n,), dtype=torch.int32, device=dev)
    b = np.ascontiguousarray(box, dtype=np.float64)
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib().dp_neighbour_list_noalloc(coords.data_ptr(), n, b.ctypes.data, float(rcut),
                                         int(nmax), j.data_ptr(), img.data_ptr(), cnt.data_ptr(), st)
    if rc:
        raise DPError(rc, lib().dp_noalloc_last_error().decode())
    return cnt, j, img


def selftest_mma(A, B, a_mn=0, b_mn=0, swap=0):
    """``dp_selftest_mma``: D = A B^T (A 128 x k, B n x k) on the tensor cores."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    n, k = B.shape
    assert A.shape == (128, k)
    D = np.zeros((128, n), np.float32)
    rc = lib().dp_selftest_mma(n, k, a_mn, b_mn, swap, A.ctypes.data, B.ctypes.data, D.ctypes.data)
    if rc:
        raise DPError(rc, "selftest_mma")
    return D


def selftest_mma_rate(n, issuers=1, reps=200):
    """``dp_selftest_mma_rate``: SM cycles per 128 x n x 16 tensor-core product."""
    out = C.c_double()
    rc = lib().dp_selftest_mma_rate(int(n), int(issuers), int(reps), C.byref(out))
    if rc:
        raise DPError(rc, "selftest_mma_rate")
    return out.value


def _dpenergy_class():
    import torch

    class DPEnergy(torch.autograd.Function):
        """E(x) through dp_compute; backward gives dE/dx = -F from the library's
        hand-written adjoint kernels (no autograd tape inside)."""

        @staticmethod
        def forward(ctx, coords, pot):
            e, f, _ = pot.compute(coords.detach().contiguous())
            if isinstance(e, float):
                e = torch.tensor(e, dtype=torch.float64)
                f = torch.as_tensor(f)
            ctx.save_for_backward(f)
            return e.reshape(())

        @staticmethod
        def backward(ctx, grad):
            (f,) = ctx.saved_tensors
            return -grad * f.to(grad.device), None

    return DPEnergy


def __getattr__(name):
    if name == "DPEnergy":
        cls = _dpenergy_class()
        globals()["DPEnergy"] = cls
        return cls
    raise AttributeError(name)
