"""Thin Python binding of librrmhd (include/rrmhd.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module only
turns torch CUDA tensors into device pointers and the current torch stream into
the cudaStream_t the library enqueues on.  There is no fallback: if
``librrmhd.so`` is missing or fails to load, importing the functions raises.

Functions carry the C names (``rrmhd_create``, ``rrmhd_imex_step``, ...);
``Context`` bundles them for one context.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librrmhd.so")

RECON = {"godunov": 0, "minmod": 1, "mc": 2, "vanleer": 3}
BC = {"outflow": 0, "periodic": 1}
PRECISION = {"fp64": 0, "fp32_bulk": 1}
STATUS = {0: "OK", 1: "EC2P", 2: "EIMPLICIT", 3: "EUNPHYS", 10: "EINVAL", 11: "ENOMEM", 12: "ECUDA",
          13: "ECAPACITY", 14: "ETIMEOUT"}


class rrmhd_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3), ("bc", C.c_int * 3)]


class rrmhd_opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("a_rad", C.c_double), ("cfl", C.c_double),
                ("pvm_eps", C.c_double), ("recon", C.c_int), ("beta_mode", C.c_int),
                ("precision", C.c_int), ("c2p_maxit", C.c_int), ("imp_maxit", C.c_int),
                ("imp_tol", C.c_double), ("lanes", C.c_int), ("pvm_k", C.c_int),
                ("pvm_products", C.c_int), ("solver", C.c_int), ("ct", C.c_int),
                ("closure", C.c_int)]


class rrmhd_tuning(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("face_block", "face_per_thread", "face_persistent", "cell_block",
                                       "cell_per_thread", "cell_persistent", "lanes")]


def tuning_dict(t):
    return {f: getattr(t, f) for f, _ in rrmhd_tuning._fields_}


def make_tuning(**kw):
    t = rrmhd_tuning(128, 1, 0, 128, 1, 0, 8)
    for k, v in kw.items():
        setattr(t, k, int(v))
    return t


class rrmhd_server_config(C.Structure):
    _fields_ = [("mem_bytes", C.c_int64), ("max_resident_cells", C.c_int64), ("max_resident", C.c_int),
                ("tuning", rrmhd_tuning)]


class rrmhd_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("steps", C.c_int32), ("cells", C.c_int64),
                ("t", C.c_double), ("submit_s", C.c_double), ("admit_s", C.c_double),
                ("done_s", C.c_double)]


class rrmhd_server_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in (
        "submitted", "admitted", "completed", "failed", "steps", "zone_updates", "relayouts",
        "resident", "resident_cells", "peak_resident_cells", "pending", "cap_cells", "cap_faces")] + [
        ("busy_s", C.c_double)]


class RRMHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# (name, restype, argtypes); names and order follow include/rrmhd.h
_VP, _I64, _I32P, _DP = C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)
_SIGNATURES = [
    ("rrmhd_default_opts", None, [C.POINTER(rrmhd_opts)]),
    ("rrmhd_create", C.c_int, [C.c_int, C.POINTER(rrmhd_grid), C.POINTER(rrmhd_opts), _VP,
                               C.POINTER(_VP)]),
    ("rrmhd_destroy", None, [_VP]),
    ("rrmhd_num_instances", C.c_int, [_VP]),
    ("rrmhd_num_cells", _I64, [_VP]),
    ("rrmhd_num_faces", _I64, [_VP, C.c_int]),
    ("rrmhd_cell_offsets", C.c_int, [_VP, C.POINTER(C.c_int64)]),
    ("rrmhd_face_offsets", C.c_int, [_VP, C.c_int, C.POINTER(C.c_int64)]),
    ("rrmhd_set_opacity", C.c_int, [_VP, _VP, _VP]),
    ("rrmhd_set_state", C.c_int, [_VP, _VP]),
    ("rrmhd_get_state", C.c_int, [_VP, _VP, _VP]),
    ("rrmhd_set_times", C.c_int, [_VP, _DP, _DP]),
    ("rrmhd_get_times", C.c_int, [_VP, _DP, _DP]),
    ("rrmhd_get_inst_status", C.c_int, [_VP, _I32P]),
    ("rrmhd_imex_step", C.c_int, [_VP, C.c_int]),
    ("rrmhd_imex_step_dt", C.c_int, [_VP, C.c_double, _DP]),
    ("rrmhd_get_first_bad_cell", C.c_int, [_VP, C.POINTER(C.c_int64)]),
    ("rrmhd_imex_step_host", C.c_int, [_VP, _VP, _VP, C.c_int]),
    ("rrmhd_checkpoint_bytes", C.c_size_t, [_VP]),
    ("rrmhd_checkpoint_save", C.c_int, [_VP, _VP]),
    ("rrmhd_checkpoint_restore", C.c_int, [_VP, _VP]),
    ("rrmhd_prim2con", C.c_int, [_VP, _VP, _VP, _I64]),
    ("rrmhd_con2prim", C.c_int, [_VP, _VP, _VP, _VP, _VP, _I64]),
    ("rrmhd_flux_sweep", C.c_int, [_VP, C.c_int, _VP]),
    ("rrmhd_flux_accumulate", C.c_int, [_VP, C.c_int, C.c_double, _VP]),
    ("rrmhd_implicit_source", C.c_int, [_VP, C.c_double, _VP, _VP, _VP, _VP, _VP]),
    ("rrmhd_prim_z", C.c_int, [_VP, _VP, _VP, _I64]),
    ("rrmhd_profile_step", C.c_int, [_VP, _DP]),
    ("rrmhd_launches_per_step", C.c_int, [_VP]),
    ("rrmhd_get_tuning", C.c_int, [_VP, C.POINTER(rrmhd_tuning)]),
    ("rrmhd_set_tuning", C.c_int, [_VP, C.POINTER(rrmhd_tuning)]),
    ("rrmhd_autotune", C.c_int, [_VP, C.c_int, C.POINTER(rrmhd_tuning), _DP]),
    ("rrmhd_set_face_field", C.c_int, [_VP, _VP]),
    ("rrmhd_get_face_field", C.c_int, [_VP, _VP]),
    ("rrmhd_probe_fp64", C.c_int, [_VP, C.c_double, _DP]),
    ("rrmhd_probe_fp64_latency", C.c_int, [_VP, _DP]),
    ("rrmhd_cfl_dt_noalloc", C.c_int, [C.POINTER(rrmhd_grid), C.POINTER(rrmhd_opts), _VP, _VP, _VP]),
    ("rrmhd_server_create", C.c_int, [C.POINTER(rrmhd_opts), C.POINTER(rrmhd_server_config),
                                      C.POINTER(_VP)]),
    ("rrmhd_server_submit", C.c_int, [_VP, C.POINTER(rrmhd_grid), _VP, _VP, _VP, C.c_double, _VP,
                                      C.POINTER(C.c_int64)]),
    ("rrmhd_server_poll", C.c_int, [_VP, C.POINTER(rrmhd_result), C.c_int]),
    ("rrmhd_server_wait_idle", C.c_int, [_VP, C.c_double]),
    ("rrmhd_server_get_stats", C.c_int, [_VP, C.POINTER(rrmhd_server_stats)]),
    ("rrmhd_server_admission", C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int,
                                         C.c_int64, C.c_int64, C.c_int]),
    ("rrmhd_server_last_error", C.c_char_p, [_VP]),
    ("rrmhd_server_destroy", None, [_VP]),
    ("rrmhd_last_error", C.c_char_p, [_VP]),
]


def lib():
    """Load librrmhd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2212_00370_gb300.build.build() (no fallback path exists)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return [s[0] for s in _SIGNATURES]


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _check(ctx, rc):
    if rc != 0:
        msg = lib().rrmhd_last_error(ctx).decode() if ctx else ""
        raise RRMHDError(rc, msg)


def make_grid(ndim, n, dx, bc=("outflow",) * 3):
    n = list(n) + [1] * (3 - len(n))
    dx = list(dx) + [1.0] * (3 - len(dx))
    bc = [BC[b] if isinstance(b, str) else int(b) for b in bc] + [0] * 3
    return rrmhd_grid(ndim, (C.c_int * 3)(*n), (C.c_double * 3)(*dx), (C.c_int * 3)(*bc[:3]))


def make_opts(**kw):
    o = rrmhd_opts()
    lib().rrmhd_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "recon" and isinstance(v, str):
            v = RECON[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "beta":
            k, v = "beta_mode", (2 if v == "radiation" else int(bool(v)))
        if k == "pvm_products" and isinstance(v, str):
            v = {"fd": 0, "tangent": 1}[v]
        if k == "solver" and isinstance(v, str):
            v = {"pvm": 0, "radhll": 1}[v]
        setattr(o, k, v)
    return o


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def rrmhd_create(grids, opts, stream=None):
    arr = (rrmhd_grid * len(grids))(*grids)
    out = C.c_void_p()
    _check(None, lib().rrmhd_create(len(grids), arr, C.byref(opts), _stream(stream), C.byref(out)))
    return out


class Context:
    """One librrmhd context: a batch of instances on one CUDA stream."""

    def __init__(self, grids, stream=None, **opts):
        import torch
        self.torch = torch
        self.opts = make_opts(**opts)
        self.ctx = rrmhd_create(grids, self.opts, stream)
        self.n_inst = lib().rrmhd_num_instances(self.ctx)
        self.ncells = lib().rrmhd_num_cells(self.ctx)

    def close(self):
        if self.ctx:
            lib().rrmhd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _t(self, *shape):
        return self.torch.empty(*shape, dtype=self.torch.float64, device="cuda")

    def num_faces(self, d):
        return lib().rrmhd_num_faces(self.ctx, d)

    def cell_offsets(self):
        off = np.zeros(self.n_inst + 1, dtype=np.int64)
        _check(self.ctx, lib().rrmhd_cell_offsets(self.ctx, off.ctypes.data_as(C.POINTER(C.c_int64))))
        return off

    def face_offsets(self, d):
        off = np.zeros(self.n_inst + 1, dtype=np.int64)
        _check(self.ctx, lib().rrmhd_face_offsets(self.ctx, d, off.ctypes.data_as(C.POINTER(C.c_int64))))
        return off

    def set_opacity(self, kappa, sigma):
        self._kappa, self._sigma = kappa.contiguous(), sigma.contiguous()  # alive until copied
        _check(self.ctx, lib().rrmhd_set_opacity(self.ctx, _ptr(self._kappa), _ptr(self._sigma)))

    def set_state(self, V):
        self._V_in = V.contiguous()
        _check(self.ctx, lib().rrmhd_set_state(self.ctx, _ptr(self._V_in)))

    def get_state(self):
        U, V = self._t(12, self.ncells), self._t(12, self.ncells)
        _check(self.ctx, lib().rrmhd_get_state(self.ctx, _ptr(U), _ptr(V)))
        return U, V

    def set_times(self, t, t_end):
        t = np.ascontiguousarray(np.broadcast_to(t, (self.n_inst,)), dtype=np.float64)
        te = np.ascontiguousarray(np.broadcast_to(t_end, (self.n_inst,)), dtype=np.float64)
        _check(self.ctx, lib().rrmhd_set_times(self.ctx, t.ctypes.data_as(_DP), te.ctypes.data_as(_DP)))

    def get_times(self):
        t = np.zeros(self.n_inst)
        dt = np.zeros(self.n_inst)
        _check(self.ctx, lib().rrmhd_get_times(self.ctx, t.ctypes.data_as(_DP), dt.ctypes.data_as(_DP)))
        return t, dt

    def inst_status(self):
        st = np.zeros(self.n_inst, dtype=np.int32)
        _check(self.ctx, lib().rrmhd_get_inst_status(self.ctx, st.ctypes.data_as(_I32P)))
        return st

    def profile_step(self):
        """One step with per-launch-group device times (ms): faces, cells, fallback, step."""
        ms = np.zeros(4)
        _check(self.ctx, lib().rrmhd_profile_step(self.ctx, ms.ctypes.data_as(_DP)))
        return ms

    def launches_per_step(self):
        return lib().rrmhd_launches_per_step(self.ctx)

    def num_face_field(self):
        return sum(self.num_faces(d) for d in range(3))

    def set_face_field(self, b):
        self._b_in = b.contiguous()
        _check(self.ctx, lib().rrmhd_set_face_field(self.ctx, _ptr(self._b_in)))

    def get_face_field(self):
        b = self._t(self.num_face_field())
        _check(self.ctx, lib().rrmhd_get_face_field(self.ctx, _ptr(b)))
        return b

    def get_tuning(self):
        t = rrmhd_tuning()
        _check(self.ctx, lib().rrmhd_get_tuning(self.ctx, C.byref(t)))
        return tuning_dict(t)

    def set_tuning(self, **kw):
        t = rrmhd_tuning()
        _check(self.ctx, lib().rrmhd_get_tuning(self.ctx, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(self.ctx, lib().rrmhd_set_tuning(self.ctx, C.byref(t)))

    def autotune(self, repeats=1):
        """Times launch shapes on real steps from the current state (restored after);
        keeps and returns the fastest (dict) and its best step time in ms."""
        t = rrmhd_tuning()
        ms = C.c_double()
        _check(self.ctx, lib().rrmhd_autotune(self.ctx, int(repeats), C.byref(t), C.byref(ms)))
        return tuning_dict(t), ms.value

    def imex_step(self, nsteps=1):
        _check(self.ctx, lib().rrmhd_imex_step(self.ctx, int(nsteps)))

    def imex_step_dt(self, dt_max):
        """One step with every instance's dt capped at dt_max; returns the dt taken."""
        dt = np.zeros(self.n_inst)
        _check(self.ctx, lib().rrmhd_imex_step_dt(self.ctx, float(dt_max), dt.ctypes.data_as(_DP)))
        return dt

    def first_bad_cell(self):
        """Per instance, the packed index of the lowest failing cell, or -1."""
        cell = np.zeros(self.n_inst, dtype=np.int64)
        _check(self.ctx, lib().rrmhd_get_first_bad_cell(self.ctx, cell.ctypes.data_as(C.POINTER(C.c_int64))))
        return cell

    def checkpoint_bytes(self):
        return int(lib().rrmhd_checkpoint_bytes(self.ctx))

    def checkpoint(self, device=True):
        """A new uint8 tensor (on the device, or pinned on the host) holding a checkpoint
        of the context; enqueued on the context's stream."""
        n = self.checkpoint_bytes()
        buf = (self.torch.empty(n, dtype=self.torch.uint8, device="cuda") if device else
               self.torch.empty(n, dtype=self.torch.uint8, pin_memory=True))
        self.checkpoint_save(buf)
        return buf

    def checkpoint_save(self, buf):
        """buf: a contiguous uint8 torch tensor of checkpoint_bytes() (device or host)."""
        assert buf.is_contiguous() and buf.dtype == self.torch.uint8 and buf.numel() >= self.checkpoint_bytes()
        _check(self.ctx, lib().rrmhd_checkpoint_save(self.ctx, C.c_void_p(buf.data_ptr())))

    def checkpoint_restore(self, buf):
        """buf: a checkpoint (uint8 tensor); the library checks that its header matches
        this context's layout, precision and ct setting (RRMHDError EINVAL if not)."""
        assert buf.is_contiguous() and buf.dtype == self.torch.uint8 and buf.numel() >= 256
        _check(self.ctx, lib().rrmhd_checkpoint_restore(self.ctx, C.c_void_p(buf.data_ptr())))

    def imex_step_host(self, V_in, V_out, nsteps=1):
        """V_in, V_out: host float64 arrays [12][ncells] (pinned torch tensors or numpy)."""
        def hp(a):
            if hasattr(a, "data_ptr"):
                assert not a.is_cuda and a.is_contiguous() and a.dtype == self.torch.float64
                return C.c_void_p(a.data_ptr())
            assert a.flags.c_contiguous and a.dtype == np.float64
            return C.c_void_p(a.ctypes.data)
        _check(self.ctx, lib().rrmhd_imex_step_host(self.ctx, hp(V_in), hp(V_out), int(nsteps)))

    def prim2con(self, V):
        n = V.shape[1]
        U = self._t(12, n)
        _check(self.ctx, lib().rrmhd_prim2con(self.ctx, _ptr(V.contiguous()), _ptr(U), n))
        return U

    def prim_z(self, V):
        n = V.shape[1]
        Z = self._t(n)
        _check(self.ctx, lib().rrmhd_prim_z(self.ctx, _ptr(V.contiguous()), _ptr(Z), n))
        return Z

    def con2prim(self, U, Zguess=None):
        n = U.shape[1]
        V = self._t(12, n)
        st = self.torch.zeros(n, dtype=self.torch.int32, device="cuda")
        _check(self.ctx, lib().rrmhd_con2prim(self.ctx, _ptr(U.contiguous()),
                                              _ptr(None if Zguess is None else Zguess.contiguous()),
                                              _ptr(V), _ptr(st), n))
        return V, st

    def flux_sweep(self, d):
        F = self._t(12, self.num_faces(d))
        _check(self.ctx, lib().rrmhd_flux_sweep(self.ctx, d, _ptr(F)))
        return F

    def flux_accumulate(self, d, dt_weight, U):
        """U -= dt_weight/dx_d (F_right - F_left) in place (U: CUDA float64 [12][ncells])."""
        _check(self.ctx, lib().rrmhd_flux_accumulate(self.ctx, int(d), float(dt_weight), _ptr(U)))
        return U

    def implicit_source(self, hdt, Ustar, Zguess=None):
        U, V = self._t(12, self.ncells), self._t(12, self.ncells)
        st = self.torch.zeros(self.ncells, dtype=self.torch.int32, device="cuda")
        _check(self.ctx, lib().rrmhd_implicit_source(
            self.ctx, float(hdt), _ptr(Ustar.contiguous()),
            _ptr(None if Zguess is None else Zguess.contiguous()), _ptr(U), _ptr(V), _ptr(st)))
        return U, V, st


def probe_fp64(target_ms=100.0, stream=None):
    """FP64-pipe rate of the current device (rrmhd_probe_fp64): thread-level FP64
    instructions per second of independent DFMA chains on every SM."""
    out = C.c_double()
    _check(None, lib().rrmhd_probe_fp64(_stream(stream), float(target_ms), C.byref(out)))
    return out.value


def probe_fp64_latency(stream=None):
    """Nanoseconds per dependent FP64 instruction of one warp (rrmhd_probe_fp64_latency)."""
    out = C.c_double()
    _check(None, lib().rrmhd_probe_fp64_latency(_stream(stream), C.byref(out)))
    return out.value


def server_admission(cells, faces, free_cells, free_faces, free_slots):
    """The server's admission rule (host only): how many requests from the head of
    the waiting queue (cells[i], faces[i] in arrival order) are admitted."""
    c = np.ascontiguousarray(cells, dtype=np.int64)
    f = np.ascontiguousarray(faces, dtype=np.int64)
    return lib().rrmhd_server_admission(c.ctypes.data_as(C.POINTER(C.c_int64)),
                                        f.ctypes.data_as(C.POINTER(C.c_int64)), len(c),
                                        int(free_cells), int(free_faces), int(free_slots))


class Server:
    """A librrmhd serving loop: requests are submitted from host arrays and run to
    completion on the current device with continuous batching."""

    def __init__(self, mem_bytes=0, max_resident_cells=0, max_resident=0, tuning=None, **opts):
        """tuning: a dict of rrmhd_tuning fields (e.g. from Context.autotune), or None."""
        self.opts = make_opts(**opts)
        cfg = rrmhd_server_config(int(mem_bytes), int(max_resident_cells), int(max_resident))
        if tuning:
            cfg.tuning = make_tuning(**tuning)
        self.srv = C.c_void_p()
        rc = lib().rrmhd_server_create(C.byref(self.opts), C.byref(cfg), C.byref(self.srv))
        if rc != 0:
            raise RRMHDError(rc, "rrmhd_server_create")
        self._out = {}  # id -> output array, alive until its result is polled

    def _check(self, rc):
        if rc != 0:
            raise RRMHDError(rc, lib().rrmhd_server_last_error(self.srv).decode())

    def submit(self, grid, V, kappa, sigma, t_end):
        """grid: rrmhd_grid; V: (12, n) float64; kappa, sigma: (n,) float64.  Returns the id."""
        V = np.ascontiguousarray(V, dtype=np.float64)
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        out = np.empty_like(V)
        rid = C.c_int64()
        self._check(lib().rrmhd_server_submit(
            self.srv, C.byref(grid), C.c_void_p(V.ctypes.data), C.c_void_p(kappa.ctypes.data),
            C.c_void_p(sigma.ctypes.data), float(t_end), C.c_void_p(out.ctypes.data), C.byref(rid)))
        self._out[rid.value] = out
        return rid.value

    def poll(self, max_results=4096):
        """Completed requests since the last poll: list of (result dict, final V)."""
        buf = (rrmhd_result * max_results)()
        k = lib().rrmhd_server_poll(self.srv, buf, max_results)
        out = []
        for r in buf[:k]:
            d = {f: getattr(r, f) for f, _ in rrmhd_result._fields_}
            out.append((d, self._out.pop(r.id)))
        return out

    def wait_idle(self, timeout_s=60.0):
        self._check(lib().rrmhd_server_wait_idle(self.srv, float(timeout_s)))

    def stats(self):
        st = rrmhd_server_stats()
        self._check(lib().rrmhd_server_get_stats(self.srv, C.byref(st)))
        return {f: getattr(st, f) for f, _ in rrmhd_server_stats._fields_}

    def close(self):
        if self.srv:
            lib().rrmhd_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
