"""Host-side argument checks of the C ABI (include/chhs.h), on the CPU.

Every case here returns before the library makes a CUDA call, so these run
without a GPU: the problem and option checks of chhs_create (Section 2's
h, eps, dt > 0, gamma >= 0 and the solver options of the Section 5
preamble), a NULL handle or server passed to every entry point, and the
argument checks of the no-allocation energy call and of the server.
"""
import ctypes
import math

import pytest

from paper_1611_02967_gb300 import build, chhs

INVALID = chhs.CHHS_ERR_INVALID_ARG
NAN, INF = float("nan"), float("inf")


@pytest.fixture(scope="module")
def L():
    build.build()
    return chhs.lib()


def _n(*ext):
    return (ctypes.c_int * 3)(*(list(ext) + [1] * (3 - len(ext))))


def _create(L, dim, n, h=0.025, eps=0.05, gamma=1.0, dt=0.005, opts=None):
    out = ctypes.c_void_p(12345)  # must be reset to NULL on every error
    s = L.chhs_create(dim, n, h, eps, gamma, dt, ctypes.byref(opts) if opts is not None else None, None,
                      ctypes.byref(out))
    return s, out.value


BAD_PROBLEMS = [
    dict(dim=1, n=_n(16, 16)),
    dict(dim=4, n=_n(16, 16, 16)),
    dict(dim=2, n=_n(1, 16)),
    dict(dim=2, n=_n(16, 0)),
    dict(dim=2, n=_n(-4, 16)),
    dict(dim=3, n=_n(16, 16, 1)),
    dict(dim=2, n=_n((1 << 20) + 2, 2)),          # an extent above 2^20
    dict(dim=3, n=_n(2048, 2048, 128)),           # 2^29 cells, above 2^28
    dict(dim=2, n=_n(16, 16), h=0.0),
    dict(dim=2, n=_n(16, 16), h=-0.1),
    dict(dim=2, n=_n(16, 16), h=NAN),
    dict(dim=2, n=_n(16, 16), h=INF),
    dict(dim=2, n=_n(16, 16), eps=0.0),
    dict(dim=2, n=_n(16, 16), eps=NAN),
    dict(dim=2, n=_n(16, 16), dt=0.0),
    dict(dim=2, n=_n(16, 16), dt=INF),
    dict(dim=2, n=_n(16, 16), gamma=-1e-300),
    dict(dim=2, n=_n(16, 16), gamma=NAN),
    dict(dim=2, n=_n(16, 16), gamma=INF),
    dict(dim=2, n=None),
]


@pytest.mark.parametrize("case", range(len(BAD_PROBLEMS)))
def test_create_rejects_bad_problem(L, case):
    s, out = _create(L, **BAD_PROBLEMS[case])
    assert s == INVALID and out is None
    kw = BAD_PROBLEMS[case]
    if kw["n"] is not None and "h" not in kw and "eps" not in kw and "dt" not in kw and "gamma" not in kw:
        # the same sizes are refused by the admission call
        assert L.chhs_workspace_bytes(kw["dim"], kw["n"], None) == 0


BAD_OPTS = [dict(nu1=0, nu2=0), dict(nu1=-1), dict(nu2=-1), dict(max_v=0), dict(coarsest=0), dict(coarsest=1),
            dict(tol=0.0),
            dict(tol=-1e-10), dict(tol=NAN), dict(precision=2), dict(precision=-1), dict(max_factor=-1.0),
            dict(max_factor=NAN), dict(max_inner=0), dict(max_inner=5)]


@pytest.mark.parametrize("case", range(len(BAD_OPTS)))
def test_create_rejects_bad_opts(L, case):
    o = chhs.default_opts(**BAD_OPTS[case])
    s, out = _create(L, 2, _n(16, 16), opts=o)
    assert s == INVALID and out is None
    assert L.chhs_workspace_bytes(2, _n(16, 16), ctypes.byref(o)) == 0


def test_create_null_out_and_null_arena(L):
    assert L.chhs_create(2, _n(16, 16), 0.025, 0.05, 1.0, 0.005, None, None, None) == INVALID
    out = ctypes.c_void_p(12345)
    s = L.chhs_create_ext(2, _n(16, 16), 0.025, 0.05, 1.0, 0.005, None, None, None, 1 << 30, ctypes.byref(out))
    assert s == INVALID
    assert L.chhs_default_opts(None) == INVALID


def test_limits_are_inclusive(L):
    # the largest accepted sizes: 2^28 cells and an extent of 2^20
    assert L.chhs_workspace_bytes(3, _n(2048, 2048, 64), None) > 0
    assert L.chhs_workspace_bytes(2, _n(1 << 20, 2), None) > 0
    assert L.chhs_workspace_bytes(2, _n(2, 2), None) > 0


# entry points taking a handle first: every one refuses NULL
HANDLE_CALLS = {
    "chhs_set_phi": (None, None, None, 0),
    "chhs_step": (None, 1, None, None),
    "chhs_step_async": (None, 1),
    "chhs_wait": (None, None, None),
    "chhs_launch_counts": (None, None, None),
    "chhs_profile_step": (None, None, None, None),
    "chhs_profile_smooth": (None, 1, None),
    "chhs_autotune": (None, 1, None),
    "chhs_mass": (None, None),
    "chhs_energy": (None, None, None),
    "chhs_dissipation": (None, None, None, None),
    "chhs_velocity": (None, None, None, None, 0),
    "chhs_get_phi": (None, None, 0),
    "chhs_get_state": (None, None, None, None, None, 0),
    "chhs_set_state": (None, None, None, None, None, 0),
    "chhs_server_submit": (None, None, None),
    "chhs_server_wait": (None, 0, 1.0),
    "chhs_server_result": (None, 0, None, None, None, None, None),
    "chhs_server_release": (None, 0),
    "chhs_server_stats": (None, None, None, None, None),
    "chhs_batch_step": (None, 1, None, None, None),
    "chhs_batch_launch_counts": (None, None, None),
    "chhs_profile_smooth32": (None, 1, None),
    "chhs_batch_profile_step": (None, None, None),
    "chhs_set_tuning": (None, None),
    "chhs_norm_checks": (None, None),
    "chhs_batch_set_tuning": (None, None),
    "chhs_batch_autotune": (None, 1, None),
}


def test_null_handle_everywhere(L):
    for name, args in HANDLE_CALLS.items():
        assert getattr(L, name)(*args) == INVALID, name
    assert L.chhs_num_levels(None) == 0
    assert L.chhs_last_error(None) == b"NULL handle"
    L.chhs_destroy(None)
    L.chhs_server_destroy(None)


def test_every_handle_entry_point_is_covered():
    # a new entry point taking a handle gets a NULL case above
    handle_free = {"chhs_default_opts", "chhs_workspace_bytes", "chhs_create", "chhs_create_ext",
                   "chhs_energy_noalloc", "chhs_server_create", "chhs_num_levels", "chhs_destroy",
                   "chhs_last_error", "chhs_server_destroy", "chhs_batch_workspace_bytes", "chhs_batch_create",
                   "chhs_batch_size", "chhs_batch_run", "chhs_batch_last_error", "chhs_batch_destroy",
                   "chhs_probe_fp64", "chhs_probe_l2"}
    assert set(chhs.EXPORTS) - handle_free == set(HANDLE_CALLS)


def test_server_create_checks(L):
    out = ctypes.c_void_p(12345)
    assert L.chhs_server_create(0, 4, 5, ctypes.byref(out)) == INVALID
    assert L.chhs_server_create(1 << 30, 0, 5, ctypes.byref(out)) == INVALID
    assert L.chhs_server_create(1 << 30, 4, 0, ctypes.byref(out)) == INVALID
    assert L.chhs_server_create(1 << 30, 4, 5, None) == INVALID


def test_energy_noalloc_checks(L):
    m, e, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    outs = (ctypes.byref(m), ctypes.byref(e), ctypes.byref(f))
    assert L.chhs_energy_noalloc(4, _n(8, 8), 0.1, 0.05, None, None, None, *outs) == INVALID
    assert L.chhs_energy_noalloc(2, None, 0.1, 0.05, None, None, None, *outs) == INVALID
    assert L.chhs_energy_noalloc(2, _n(8, 8), 0.1, 0.05, None, None, None, *outs) == INVALID  # phi NULL


def test_status_names_match_header():
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "include", "chhs.h")).read()
    vals = {k: int(v) for k, v in re.findall(r"\b(CHHS_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", src)}
    assert vals == {v: k for k, v in chhs.STATUS_NAMES.items()}
    assert not math.isnan(chhs.default_opts().tol)


def _gpu_present():
    import torch
    return torch.cuda.is_available()


@pytest.mark.skipif(_gpu_present(), reason="passes addresses that are not device memory")
def test_create_ext_arena_checks(L):
    # misaligned or too small: refused before any CUDA call, so these
    # addresses (never dereferenced) are safe here
    need = L.chhs_workspace_bytes(2, _n(16, 16), None)
    out = ctypes.c_void_p(12345)
    args = (2, _n(16, 16), 0.025, 0.05, 1.0, 0.005, None, None)
    assert L.chhs_create_ext(*args, ctypes.c_void_p(0x10010), need, ctypes.byref(out)) == INVALID
    assert out.value is None
    assert L.chhs_create_ext(*args, ctypes.c_void_p(0x10000), need - 1, ctypes.byref(out)) == chhs.CHHS_ERR_OOM
    assert out.value is None


@pytest.mark.skipif(_gpu_present(), reason="checks the behaviour without a usable GPU")
def test_no_gpu_fails_loudly(L):
    # valid arguments, no GPU: CHHS_ERR_CUDA and no handle, never a CPU path
    s, out = _create(L, 2, _n(16, 16))
    assert s == chhs.CHHS_ERR_CUDA and out is None
    with pytest.raises(chhs.ChhsError) as e:
        chhs.Run((16, 16), 0.025, 0.05, 1.0, 0.005)
    assert e.value.status == chhs.CHHS_ERR_CUDA
    sv = ctypes.c_void_p(12345)
    assert L.chhs_server_create(1 << 30, 4, 5, ctypes.byref(sv)) == chhs.CHHS_ERR_CUDA
    assert sv.value is None


def test_binding_buffer_checks():
    # the binding's marshalling of host buffers (chhs._buf): what it copies,
    # what it refuses
    import numpy as np
    import torch

    a = np.arange(12, dtype=np.float64).reshape(3, 4)
    p, dev, keep = chhs._buf(a, 12)
    assert dev == 0 and keep is a and p.value == a.ctypes.data  # no copy
    f32 = a.astype(np.float32)
    p, dev, keep = chhs._buf(f32, 12)
    assert keep.dtype == np.float64 and np.array_equal(keep, a)  # converted copy for inputs
    with pytest.raises(ValueError):
        chhs._buf(f32, 12, writable=True)  # an output must be written in place
    with pytest.raises(ValueError):
        chhs._buf(a.T, 12, writable=True)  # not C-contiguous
    with pytest.raises(ValueError):
        chhs._buf(a, 13)
    t = torch.zeros(12, dtype=torch.float64)
    p, dev, keep = chhs._buf(t, 12)
    assert dev == 0 and p.value == t.data_ptr()
    with pytest.raises(ValueError):
        chhs._buf(torch.zeros(12, dtype=torch.float32), 12)
    with pytest.raises(ValueError):
        chhs._buf(torch.zeros(24, dtype=torch.float64)[::2], 12)  # strided view
    assert chhs._buf(None, 12) == (None, 0, None)


def _descs(specs):
    arr = (chhs.chhs_run_desc * len(specs))()
    for q, (dim, n, h, eps, gamma, dt) in enumerate(specs):
        arr[q] = chhs.chhs_run_desc(dim, (ctypes.c_int * 3)(*n), h, eps, gamma, dt)
    return arr


def test_batch_arguments_checked_before_any_cuda_call(L):
    good = (2, (64, 64, 1), 0.025, 0.05, 1.0, 0.005)
    mixed = chhs.default_opts(precision=1)
    one = _descs([good])
    assert L.chhs_batch_workspace_bytes(1, one, ctypes.byref(mixed)) > 0
    assert L.chhs_batch_workspace_bytes(1, one, None) > 0  # NULL opts: the mixed-precision defaults
    # no runs, runs of two dimensions, a bad run, the double-precision form
    assert L.chhs_batch_workspace_bytes(0, one, None) == 0
    assert L.chhs_batch_workspace_bytes(2, _descs([good, (3, (16, 16, 16), 0.1, 0.05, 1.0, 0.005)]), None) == 0
    assert L.chhs_batch_workspace_bytes(2, _descs([good, (2, (64, 64, 1), -0.1, 0.05, 1.0, 0.005)]), None) == 0
    assert L.chhs_batch_workspace_bytes(1, one, ctypes.byref(chhs.default_opts(precision=0))) == 0
    out = ctypes.c_void_p(1234)
    assert L.chhs_batch_create(0, one, None, None, ctypes.byref(out)) == INVALID and not out.value
    assert L.chhs_batch_create(1, one, None, None, None) == INVALID
    # the batch's hierarchies are the runs' own, summed
    two = _descs([good, (2, (128, 32, 1), 0.025, 0.05, 1.0, 0.005)])
    w1 = L.chhs_workspace_bytes(2, (ctypes.c_int * 3)(64, 64, 1), ctypes.byref(mixed))
    w2 = L.chhs_workspace_bytes(2, (ctypes.c_int * 3)(128, 32, 1), ctypes.byref(mixed))
    assert L.chhs_batch_workspace_bytes(2, two, None) >= w1 + w2
    # NULL batch
    assert L.chhs_batch_step(None, 1, None, None, None) == INVALID
    assert L.chhs_batch_size(None) == 0 and L.chhs_batch_run(None, 0) is None
    L.chhs_batch_destroy(None)


def test_probe_argument_checks(L):
    """The measurement probes refuse bad arguments before any CUDA call."""
    g = ctypes.c_double()
    assert L.chhs_probe_fp64(None) == INVALID
    assert L.chhs_probe_l2(1 << 24, 10, None) == INVALID
    assert L.chhs_probe_l2(1 << 24, 0, ctypes.byref(g)) == INVALID
    assert L.chhs_probe_l2(1000, 10, ctypes.byref(g)) == INVALID
    assert L.chhs_probe_l2(1 << 31, 10, ctypes.byref(g)) == INVALID
