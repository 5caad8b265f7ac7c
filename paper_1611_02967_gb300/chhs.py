"""Thin ctypes binding of the C ABI in ``include/chhs.h`` (``libchhs.so``).

Argument marshalling only: every step of the solve runs in the CUDA library.
Functions keep the C names (``chhs_create``, ``chhs_step``, ``chhs_mass``,
``chhs_energy`` ...); ``Run`` wraps a handle for convenience.  Arrays are
numpy float64 (host) or CUDA torch float64 tensors (device), C-contiguous,
indexed [y, x] or [z, y, x] (x fastest).

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1611_02967_gb300.build``); loading raises if it is missing.
There is no fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchhs.so")

CHHS_OK, CHHS_ERR_INVALID_ARG, CHHS_ERR_OOM, CHHS_ERR_CUDA, CHHS_ERR_NOT_CONVERGED, CHHS_ERR_DIVERGED = range(6)
STATUS_NAMES = {0: "CHHS_OK", 1: "CHHS_ERR_INVALID_ARG", 2: "CHHS_ERR_OOM", 3: "CHHS_ERR_CUDA",
                4: "CHHS_ERR_NOT_CONVERGED", 5: "CHHS_ERR_DIVERGED"}

EXPORTS = ["chhs_default_opts", "chhs_workspace_bytes", "chhs_create", "chhs_create_ext", "chhs_set_phi",
           "chhs_step", "chhs_step_async", "chhs_wait", "chhs_launch_counts", "chhs_profile_step",
           "chhs_mass", "chhs_energy", "chhs_get_phi", "chhs_get_state", "chhs_set_state",
           "chhs_num_levels", "chhs_destroy", "chhs_last_error", "chhs_energy_noalloc", "chhs_dissipation",
           "chhs_server_create", "chhs_server_submit", "chhs_server_wait", "chhs_server_result",
           "chhs_server_release", "chhs_server_stats", "chhs_server_destroy", "chhs_profile_smooth", "chhs_velocity",
           "chhs_autotune", "chhs_batch_workspace_bytes", "chhs_batch_create", "chhs_batch_size", "chhs_batch_run",
           "chhs_batch_step", "chhs_batch_launch_counts", "chhs_batch_last_error", "chhs_batch_destroy",
           "chhs_profile_smooth32", "chhs_probe_fp64", "chhs_probe_l2", "chhs_batch_profile_step", "chhs_set_tuning",
           "chhs_norm_checks", "chhs_batch_set_tuning", "chhs_batch_autotune"]

# kernel kinds of chhs_profile_step
kTileThreads = 512  # threads of a 2D tile (the batch's fixed tile launch)

K_NAMES = ["smooth", "residual_restrict", "coarse_rhs", "prolong", "tail", "norm", "frame", "smooth_finest"]


class chhs_opts(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_v", ctypes.c_int),
                ("coarsest", ctypes.c_int), ("tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("max_factor", ctypes.c_double), ("coarsest_f64", ctypes.c_int), ("f64_residual", ctypes.c_int),
                ("max_inner", ctypes.c_int)]


class chhs_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("eps", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dt", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("precision", ctypes.c_int), ("phi0", ctypes.c_void_p), ("phi_prev", ctypes.c_void_p)]


class chhs_run_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("eps", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dt", ctypes.c_double)]


class Tuning(ctypes.Structure):
    """chhs_tuning (include/chhs.h)."""
    _fields_ = [("tail_cells", ctypes.c_int), ("split_threads", ctypes.c_int), ("tile_threads", ctypes.c_int),
                ("coarse_nu1", ctypes.c_int), ("coarse_nu2", ctypes.c_int), ("tile_w", ctypes.c_int),
                ("tile_h", ctypes.c_int), ("norm_f64_per8", ctypes.c_int), ("small_tile_w", ctypes.c_int),
                ("small_tile_h", ctypes.c_int), ("small_tile_threads", ctypes.c_int), ("quad_passes", ctypes.c_int),
                ("ms_per_step", ctypes.c_double)]


class ChhsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None
_vp, _dp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)


def lib():
    """Load libchhs.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libchhs.so not built: run python -m paper_1611_02967_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        optp = ctypes.POINTER(chhs_opts)
        sig = {
            "chhs_default_opts": (i, [optp]),
            "chhs_workspace_bytes": (sz, [i, _ip, optp]),
            "chhs_create": (i, [i, _ip, d, d, d, d, optp, _vp, ctypes.POINTER(_vp)]),
            "chhs_create_ext": (i, [i, _ip, d, d, d, d, optp, _vp, _vp, sz, ctypes.POINTER(_vp)]),
            "chhs_set_phi": (i, [_vp, _vp, _vp, i]),
            "chhs_step": (i, [_vp, i, _ip, _dp]),
            "chhs_step_async": (i, [_vp, i]),
            "chhs_wait": (i, [_vp, _ip, _dp]),
            "chhs_launch_counts": (i, [_vp, _ip, _ip]),
            "chhs_norm_checks": (i, [_vp, _ip]),
            "chhs_profile_step": (i, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong), _dp]),
            "chhs_mass": (i, [_vp, _dp]),
            "chhs_energy": (i, [_vp, _dp, _dp]),
            "chhs_dissipation": (i, [_vp, _dp, _dp, _dp]),
            "chhs_server_create": (i, [sz, i, i, ctypes.POINTER(_vp)]),
            "chhs_server_submit": (i, [_vp, ctypes.POINTER(chhs_request), ctypes.POINTER(ctypes.c_longlong)]),
            "chhs_server_wait": (i, [_vp, ctypes.c_longlong, d]),
            "chhs_server_result": (i, [_vp, ctypes.c_longlong, _ip, _ip, _ip, _vp, _dp]),
            "chhs_server_release": (i, [_vp, ctypes.c_longlong]),
            "chhs_server_stats": (i, [_vp, _ip, _ip, _ip, ctypes.POINTER(sz)]),
            "chhs_server_destroy": (None, [_vp]),
            "chhs_profile_smooth": (i, [_vp, i, _dp]),
            "chhs_velocity": (i, [_vp, _dp, _dp, _dp, i]),
            "chhs_autotune": (i, [_vp, i, ctypes.c_void_p]),
            "chhs_get_phi": (i, [_vp, _vp, i]),
            "chhs_get_state": (i, [_vp, _vp, _vp, _vp, _vp, i]),
            "chhs_set_state": (i, [_vp, _vp, _vp, _vp, _vp, i]),
            "chhs_num_levels": (i, [_vp]),
            "chhs_destroy": (None, [_vp]),
            "chhs_last_error": (ctypes.c_char_p, [_vp]),
            "chhs_energy_noalloc": (i, [i, _ip, d, d, _vp, _vp, _vp, _dp, _dp, _dp]),
            "chhs_batch_workspace_bytes": (sz, [i, ctypes.POINTER(chhs_run_desc), optp]),
            "chhs_batch_create": (i, [i, ctypes.POINTER(chhs_run_desc), optp, _vp, ctypes.POINTER(_vp)]),
            "chhs_batch_size": (i, [_vp]),
            "chhs_batch_run": (_vp, [_vp, i]),
            "chhs_batch_step": (i, [_vp, i, _ip, _ip, _dp]),
            "chhs_batch_launch_counts": (i, [_vp, _ip, _ip]),
            "chhs_batch_last_error": (ctypes.c_char_p, [_vp]),
            "chhs_batch_destroy": (None, [_vp]),
            "chhs_profile_smooth32": (i, [_vp, i, _dp]),
            "chhs_probe_fp64": (i, [_dp]),
            "chhs_probe_l2": (i, [ctypes.c_size_t, i, _dp]),
            "chhs_batch_profile_step": (i, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
            "chhs_set_tuning": (i, [_vp, ctypes.c_void_p]),
            "chhs_batch_set_tuning": (i, [_vp, ctypes.c_void_p]),
            "chhs_batch_autotune": (i, [_vp, i, ctypes.c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_opts(**kw):
    o = chhs_opts()
    lib().chhs_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dims(shape):
    n = list(shape[::-1]) + [1] * (3 - len(shape))
    return len(shape), (ctypes.c_int * 3)(*n)


def _buf(a, n, writable=False):
    """(pointer, on_device, keepalive) for a numpy array or CUDA torch tensor of n doubles."""
    if a is None:
        return None, 0, None
    mod = type(a).__module__
    if mod.startswith("torch"):
        if a.dtype.__repr__() != "torch.float64" or not a.is_contiguous() or a.numel() != n:
            raise ValueError("need a contiguous float64 tensor of %d elements" % n)
        return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0), a
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags.c_contiguous or arr.size != n:
        if writable:
            raise ValueError("need a C-contiguous float64 array of %d elements" % n)
        arr = np.ascontiguousarray(arr, dtype=np.float64)
        if arr.size != n:
            raise ValueError("need %d elements" % n)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def energy_noalloc(phi, psi, h, eps, stream=None):
    """(mass, E_h(phi), F_h(phi, psi)) of CUDA float64 tensors, computed with
    the library's fixed scratch array and no device allocation."""
    n = int(np.prod(phi.shape))
    p0, dev0, _ = _buf(phi, n)
    p1, dev1, _ = _buf(psi, n)
    if not dev0 or (psi is not None and not dev1):
        raise ValueError("phi and psi must be CUDA tensors")
    dim, nn = _dims(tuple(phi.shape))
    m, E, F = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    s = lib().chhs_energy_noalloc(dim, nn, float(h), float(eps), p0, p1, ctypes.c_void_p(stream) if stream else None,
                                  ctypes.byref(m), ctypes.byref(E), ctypes.byref(F))
    if s != CHHS_OK:
        raise ChhsError(s, "chhs_energy_noalloc failed")
    return m.value, E.value, F.value


def workspace_bytes(shape, opts=None):
    dim, n = _dims(shape)
    return lib().chhs_workspace_bytes(dim, n, ctypes.byref(opts) if opts is not None else None)


class Run:
    """One CHHS run (a chhs_t handle)."""

    @classmethod
    def _member(cls, handle, shape, h, eps, gamma, dt):
        """A run owned by a Batch (chhs_batch_run): usable, never destroyed here."""
        self = cls.__new__(cls)
        self.shape = tuple(int(x) for x in shape)
        self.ncell = int(np.prod(self.shape))
        self.h, self.eps, self.gamma, self.dt = float(h), float(eps), float(gamma), float(dt)
        self._arena = None
        self.handle = ctypes.c_void_p(handle)
        self._member_of_batch = True
        return self

    def __init__(self, shape, h, eps, gamma, dt, opts=None, stream=None, arena=None):
        self.shape = tuple(int(x) for x in shape)
        self.ncell = int(np.prod(self.shape))
        self.h, self.eps, self.gamma, self.dt = float(h), float(eps), float(gamma), float(dt)
        dim, n = _dims(self.shape)
        handle = ctypes.c_void_p()
        optp = ctypes.byref(opts) if opts is not None else None
        st = ctypes.c_void_p(stream) if stream else None
        self._arena = arena
        if arena is not None:
            s = lib().chhs_create_ext(dim, n, self.h, self.eps, self.gamma, self.dt, optp, st,
                                      ctypes.c_void_p(arena.data_ptr()), arena.numel() * arena.element_size(),
                                      ctypes.byref(handle))
        else:
            s = lib().chhs_create(dim, n, self.h, self.eps, self.gamma, self.dt, optp, st, ctypes.byref(handle))
        if s != CHHS_OK:
            raise ChhsError(s, "chhs_create failed")
        self.handle = handle

    def _check(self, s):
        if s != CHHS_OK:
            raise ChhsError(s, lib().chhs_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            if not getattr(self, "_member_of_batch", False):
                lib().chhs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def num_levels(self):
        return lib().chhs_num_levels(self.handle)

    def set_phi(self, phi0, phi_prev=None):
        p0, dev0, k0 = _buf(phi0, self.ncell)
        p1, dev1, k1 = _buf(phi_prev, self.ncell)
        if phi_prev is not None and dev0 != dev1:
            raise ValueError("phi0 and phi_prev must both be host or both be device")
        self._check(lib().chhs_set_phi(self.handle, p0, p1, dev0))

    def step(self, nsteps=1, check=True):
        """Advance nsteps; returns (status, total V-cycles, last residual)."""
        v = ctypes.c_int(0)
        r = ctypes.c_double(0.0)
        s = lib().chhs_step(self.handle, int(nsteps), ctypes.byref(v), ctypes.byref(r))
        if check:
            self._check(s)
        return s, v.value, r.value

    def step_async(self, nsteps=1):
        self._check(lib().chhs_step_async(self.handle, int(nsteps)))

    def wait(self, check=True):
        v = ctypes.c_int(0)
        r = ctypes.c_double(0.0)
        s = lib().chhs_wait(self.handle, ctypes.byref(v), ctypes.byref(r))
        if check:
            self._check(s)
        return s, v.value, r.value

    def launch_counts(self):
        """(kernels per V-cycle, kernels per step outside the V-cycle loop)."""
        a = ctypes.c_int(0)
        b = ctypes.c_int(0)
        self._check(lib().chhs_launch_counts(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def norm_checks(self):
        """Stopping norms after V-cycles in the last completed step call."""
        c = ctypes.c_int(0)
        self._check(lib().chhs_norm_checks(self.handle, ctypes.byref(c)))
        return c.value

    def profile_step(self, acc=None):
        """One step launched kernel by kernel with events; accumulates into
        acc = {kind: [ms, launches, units]} and returns it."""
        n = len(K_NAMES)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_longlong * n)()
        un = (ctypes.c_double * n)()
        self._check(lib().chhs_profile_step(self.handle, ms, la, un))
        acc = acc if acc is not None else {k: [0.0, 0, 0.0] for k in K_NAMES}
        for q, k in enumerate(K_NAMES):
            acc[k][0] += ms[q]
            acc[k][1] += la[q]
            acc[k][2] += un[q]
        return acc

    def profile_smooth(self, npasses=100):
        """Average ms of one finest-level double-precision smoother pass, timed
        back to back (call after a converged step)."""
        ms = ctypes.c_double(0.0)
        self._check(lib().chhs_profile_smooth(self.handle, int(npasses), ctypes.byref(ms)))
        return ms.value

    def profile_smooth32(self, npasses=100):
        """Average ms of the mixed form's single-precision finest-level
        smoothing launch (2D: the pre-smoothing tile launch; 3D: one colour
        pass), timed back to back."""
        ms = ctypes.c_double(0.0)
        self._check(lib().chhs_profile_smooth32(self.handle, int(npasses), ctypes.byref(ms)))
        return ms.value

    def velocity(self):
        """Face velocities of the last accepted step (Eq. 2.3): array (dim,) +
        shape, [a][c] on the face between cell c and its +a neighbour."""
        dim = len(self.shape)
        u = np.zeros((dim,) + tuple(self.shape))
        ptr = [u[a].ctypes.data_as(_dp) for a in range(dim)] + [None] * (3 - dim)
        self._check(lib().chhs_velocity(self.handle, ptr[0], ptr[1], ptr[2], 0))
        return u

    def autotune(self, trial_steps=3):
        """chhs_autotune: pick this run's launch shapes by timing its own steps
        (the state is left as it was).  Returns the chosen setting."""
        t = Tuning()
        self._check(lib().chhs_autotune(self.handle, int(trial_steps), ctypes.byref(t)))
        return dict(tail_cells=t.tail_cells, split_threads=t.split_threads, tile_threads=t.tile_threads,
                    coarse_nu1=t.coarse_nu1, coarse_nu2=t.coarse_nu2, tile_w=t.tile_w, tile_h=t.tile_h,
                    norm_f64_per8=t.norm_f64_per8, small_tile=(t.small_tile_w, t.small_tile_h,
                                                                 t.small_tile_threads),
                    quad_passes=t.quad_passes, ms_per_step=t.ms_per_step)

    def set_tuning(self, tail_cells, split_threads, tile_threads, coarse_nu1, coarse_nu2, tile_w=32, tile_h=32,
                   norm_f64_per8=3, small_tile=(16, 8, 256), quad_passes=1):
        """chhs_set_tuning: apply launch shapes and coarse sweep counts
        (tile_w, tile_h, tile_threads: the 2D mixed form's tiles on levels of
        at least 512 x 256 cells; small_tile: (width, height, threads) on the
        smaller levels; quad_passes: the 3D mixed form's colour passes on four
        cells per thread (1) or one (0))."""
        cw, ch, ct = small_tile
        t = Tuning(int(tail_cells), int(split_threads), int(tile_threads), int(coarse_nu1), int(coarse_nu2),
                   int(tile_w), int(tile_h), int(norm_f64_per8), int(cw), int(ch), int(ct), int(quad_passes), 0.0)
        self._check(lib().chhs_set_tuning(self.handle, ctypes.byref(t)))

    def mass(self):
        m = ctypes.c_double(0.0)
        self._check(lib().chhs_mass(self.handle, ctypes.byref(m)))
        return m.value

    def energy(self):
        E = ctypes.c_double(0.0)
        F = ctypes.c_double(0.0)
        self._check(lib().chhs_energy(self.handle, ctypes.byref(E), ctypes.byref(F)))
        return E.value, F.value

    def dissipation(self):
        """(||grad_h mu||^2, ||u||^2, max |div_h u|) of the last accepted step."""
        a, b, c = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._check(lib().chhs_dissipation(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def get_phi(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, dev, _ = _buf(out, self.ncell, writable=True)
        self._check(lib().chhs_get_phi(self.handle, p, dev))
        return out

    def get_state(self):
        """(phi^m, phi^{m-1}, mu, p) as host arrays."""
        outs = [np.empty(self.shape) for _ in range(4)]
        ptrs = [_buf(o, self.ncell, writable=True)[0] for o in outs]
        self._check(lib().chhs_get_state(self.handle, *ptrs, 0))
        return tuple(outs)

    def set_state(self, phi, phi_prev, mu=None, p=None):
        bufs = [_buf(a, self.ncell) for a in (phi, phi_prev, mu, p)]
        devs = {b[1] for b in bufs if b[0] is not None}
        if len(devs) > 1:
            raise ValueError("mixed host and device buffers")
        self._check(lib().chhs_set_state(self.handle, *[b[0] for b in bufs], devs.pop() if devs else 0))


class Server:
    """The request loop of the C ABI (chhs_server_*): continuous batching of
    independent runs on one GPU."""

    def __init__(self, pool_bytes, max_active=16, steps_per_slice=5):
        h = ctypes.c_void_p()
        st = lib().chhs_server_create(int(pool_bytes), int(max_active), int(steps_per_slice), ctypes.byref(h))
        if st != CHHS_OK:
            raise ChhsError(st, "chhs_server_create failed")
        self.handle = h
        self.shapes = {}

    def submit(self, shape, h, eps, gamma, dt, nsteps, phi0, precision=0, phi_prev=None):
        shape = tuple(int(x) for x in shape)
        n = int(np.prod(shape))
        dim, nn = _dims(shape)
        p0, dev0, k0 = _buf(phi0, n)
        p1, dev1, k1 = _buf(phi_prev, n)
        if dev0 or dev1:
            raise ValueError("server requests take host arrays")
        r = chhs_request(dim, nn, float(h), float(eps), float(gamma), float(dt), int(nsteps), int(precision),
                         p0, p1)
        rid = ctypes.c_longlong(0)
        st = lib().chhs_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid))
        if st != CHHS_OK:
            raise ChhsError(st, "chhs_server_submit failed")
        self.shapes[rid.value] = shape
        return rid.value

    def wait(self, rid, timeout=60.0):
        return lib().chhs_server_wait(self.handle, ctypes.c_longlong(rid), float(timeout)) == CHHS_OK

    def result(self, rid, with_phi=True):
        """dict(done, status, vcycles, phi, t_submit, t_admit, t_done) of a run."""
        done, status, v = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        times = (ctypes.c_double * 3)()
        phi = np.empty(self.shapes[rid]) if with_phi else None
        st = lib().chhs_server_result(self.handle, ctypes.c_longlong(rid), ctypes.byref(done), ctypes.byref(status),
                                      ctypes.byref(v), ctypes.c_void_p(phi.ctypes.data) if with_phi else None, times)
        if st != CHHS_OK:
            raise ChhsError(st, "chhs_server_result failed")
        if not done.value:
            return dict(done=False)
        return dict(done=True, status=status.value, vcycles=v.value, phi=phi, t_submit=times[0],
                    t_admit=times[1], t_done=times[2])

    def release(self, rid):
        lib().chhs_server_release(self.handle, ctypes.c_longlong(rid))
        self.shapes.pop(rid, None)

    def stats(self):
        q, a, d = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        used = ctypes.c_size_t(0)
        lib().chhs_server_stats(self.handle, ctypes.byref(q), ctypes.byref(a), ctypes.byref(d), ctypes.byref(used))
        return dict(queued=q.value, active=a.value, done=d.value, pool_in_use=used.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().chhs_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many runs stepped by one graph of batched launches (chhs_batch_*).

    runs: a list of (shape, h, eps, gamma, dt), all 2D or all 3D.  The
    batch uses the mixed-precision form; opts (chhs_opts) defaults to it."""

    def __init__(self, runs, opts=None, stream=None):
        self.specs = [(tuple(int(x) for x in r[0]),) + tuple(float(v) for v in r[1:]) for r in runs]
        descs = (chhs_run_desc * len(runs))()
        for q, (shape, h, eps, gamma, dt) in enumerate(self.specs):
            dim, n = _dims(shape)
            descs[q] = chhs_run_desc(dim, n, h, eps, gamma, dt)
        self._descs = descs
        if opts is None:
            opts = default_opts(precision=1)
        h = ctypes.c_void_p()
        st = lib().chhs_batch_create(len(runs), descs, ctypes.byref(opts), ctypes.c_void_p(stream) if stream else None,
                                     ctypes.byref(h))
        if st != CHHS_OK:
            raise ChhsError(st, "chhs_batch_create failed")
        self.handle = h
        self.runs = [Run._member(lib().chhs_batch_run(h, q), *self.specs[q]) for q in range(len(runs))]

    def __len__(self):
        return lib().chhs_batch_size(self.handle)

    def step(self, nsteps=1, check=True):
        """Advance every run nsteps; returns (statuses, V-cycles, residuals) per run."""
        n = len(self.runs)
        s_, v_, r_ = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_double * n)()
        st = lib().chhs_batch_step(self.handle, int(nsteps), s_, v_, r_)
        if check and st != CHHS_OK:
            raise ChhsError(st, lib().chhs_batch_last_error(self.handle).decode())
        return list(s_), list(v_), list(r_)

    def profile_step(self, acc=None):
        """One step of every run launched kernel by kernel with events;
        accumulates {kind: [ms, launches]}."""
        n = len(K_NAMES)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_longlong * n)()
        st = lib().chhs_batch_profile_step(self.handle, ms, la)
        if st != CHHS_OK:
            raise ChhsError(st, lib().chhs_batch_last_error(self.handle).decode())
        acc = acc if acc is not None else {k: [0.0, 0] for k in K_NAMES}
        for q, k in enumerate(K_NAMES):
            acc[k][0] += ms[q]
            acc[k][1] += la[q]
        return acc

    def launch_counts(self):
        a, b = ctypes.c_int(0), ctypes.c_int(0)
        lib().chhs_batch_launch_counts(self.handle, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def _check(self, st, what):
        if st != CHHS_OK:
            raise ChhsError(st, "%s: %s" % (what, lib().chhs_batch_last_error(self.handle).decode()))

    def set_tuning(self, tail_cells, coarse_nu1, coarse_nu2, norm_f64_per8=3, tile=(32, 16, 512)):
        """chhs_batch_set_tuning: tail size, coarse sweep counts and the norm's
        FP64 share for every run, and (width, height, threads) of the per-run
        tile launches of large 2D levels; rebuilds the batch's graph."""
        tw, th, tt = tile
        t = Tuning(int(tail_cells), 0, int(tt), int(coarse_nu1), int(coarse_nu2), int(tw), int(th), int(norm_f64_per8),
                   32, 16, kTileThreads, 0, 0.0)
        self._check(lib().chhs_batch_set_tuning(self.handle, ctypes.byref(t)), "chhs_batch_set_tuning")

    def autotune(self, trial_steps=2):
        """chhs_batch_autotune: pick the batch's tail size and coarse sweep
        counts by timing its own steps (every run's state is left as it was)."""
        t = Tuning()
        self._check(lib().chhs_batch_autotune(self.handle, int(trial_steps), ctypes.byref(t)), "chhs_batch_autotune")
        return dict(tail_cells=t.tail_cells, coarse_nu1=t.coarse_nu1, coarse_nu2=t.coarse_nu2,
                    norm_f64_per8=t.norm_f64_per8, tile=(t.tile_w, t.tile_h, t.tile_threads),
                    ms_per_step=t.ms_per_step)

    def close(self):
        if getattr(self, "handle", None):
            for r in self.runs:
                r.handle = None
            lib().chhs_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_l2(nbytes=48 << 20, passes=50):
    """Measured L2 read bandwidth of the current device in GB/s (a buffer of
    nbytes read passes times with L1-bypassing loads)."""
    g = ctypes.c_double(0.0)
    st = lib().chhs_probe_l2(int(nbytes), int(passes), ctypes.byref(g))
    if st != CHHS_OK:
        raise ChhsError(st, "chhs_probe_l2 failed")
    return g.value


def probe_fp64():
    """Measured FP64 FMA throughput of the current device in TFLOP/s."""
    t = ctypes.c_double(0.0)
    st = lib().chhs_probe_fp64(ctypes.byref(t))
    if st != CHHS_OK:
        raise ChhsError(st, "chhs_probe_fp64 failed")
    return t.value
