"""GB300 library for the adaptively compressed exchange (ACE) operator.

The data-parallel hot path of the MTACE / s-MTACE schemes of arXiv:2110.07670
(Sections 2.1-2.2, Eq. 1-5): pair densities, their FFT Poisson solves, the
exchange accumulation W = alpha V_X Phi, M = Phi^T W, the Cholesky factor of
-M, the ACE vectors xi = W L^-T and the inner-step apply K psi = -xi (xi^T psi).

All arithmetic runs in the CUDA library libace_gb300.so (C ABI in
include/ace.h).  This module only marshals arguments: PyTorch tensors supply
device memory and the current CUDA stream.  There is no CPU fallback; calls
fail loudly when the library is missing.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ACE_FP64 = 0
ACE_MIXED = 1
_ERRORS = {-1: "ACE_ERR_INVALID_ARG", -2: "ACE_ERR_GRID_TOO_SMALL", -3: "ACE_ERR_NOT_POSDEF", -4: "ACE_ERR_OOM",
           -5: "ACE_ERR_CUDA", -6: "ACE_ERR_TIMEOUT"}
SYMBOLS = ("ace_plan_create", "ace_plan_destroy", "ace_gvec", "ace_build", "ace_apply", "hfx_apply_exact",
           "ace_last_intermediates", "ace_set_timing", "ace_get_stats", "ace_last_error", "ace_apply_noalloc",
           "ace_build_batched", "ace_save", "ace_load", "ace_build_pairs", "ace_build_finish",
           "ace_plan_config", "ace_overlap_screen", "ace_build_async", "ace_build_result",
           "ace_check_timeout_path", "ace_scdm", "ace_apply_energy", "ace_plan_tuning", "ace_plan_radix", "ace_apply_prepare")

_lib = None


class AceError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class _System(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("psi_G", ctypes.c_void_p), ("n_occ", ctypes.c_int),
                ("alpha", ctypes.c_double), ("pair_row_ptr", ctypes.c_void_p), ("pair_col", ctypes.c_void_p),
                ("xi", ctypes.c_void_p), ("E_x", ctypes.c_double), ("status", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("pair_batch", ctypes.c_int), ("kernels", ctypes.c_int), ("pair_streams", ctypes.c_int),
                ("pair_variant", ctypes.c_int), ("coulomb_rc", ctypes.c_double), ("coulomb_g0", ctypes.c_int)]


STAT_FIELDS = ("orbitals_ms", "pair_fwd_ms", "pair_coulomb_ms", "pair_inv_ms", "w_to_g_ms", "gram_ms", "factor_ms",
               "xi_ms", "energy_ms", "total_ms")


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in STAT_FIELDS] + [("pair_transforms", ctypes.c_longlong),
                                                               ("launches", ctypes.c_longlong),
                                                               ("pair_wall_ms", ctypes.c_double)]


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libace_gb300.so (raises when it is missing unless asked to build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with paper_2110_07670_gb300.build.build_library()")
        _build.build_library()
    lib = ctypes.CDLL(path)
    P, i32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ace_plan_create.argtypes = [ctypes.POINTER(P), P, P, f64, i32, i32, ctypes.POINTER(_Opts)]
    lib.ace_plan_destroy.argtypes = [P]
    lib.ace_plan_destroy.restype = None
    lib.ace_gvec.argtypes = [P, ctypes.POINTER(i32), P]
    lib.ace_build.argtypes = [P, P, i32, f64, P, P, P, ctypes.POINTER(f64), P]
    lib.ace_apply.argtypes = [P, P, i32, P, i32, P, P]
    lib.ace_apply_energy.argtypes = [P, P, i32, P, i32, ctypes.POINTER(f64), P]
    lib.ace_build_pairs.argtypes = [P, P, i32, f64, P, P, P, ctypes.POINTER(f64), P]
    lib.ace_build_finish.argtypes = [P, P, i32, P, P, P]
    lib.ace_build_async.argtypes = [P, P, i32, f64, P, P, P, P]
    lib.ace_check_timeout_path.argtypes = [P, i32, P]
    lib.ace_build_result.argtypes = [P, ctypes.POINTER(f64), P]
    lib.ace_overlap_screen.argtypes = [P, P, i32, f64, P, P, ctypes.POINTER(i32), P, P]
    lib.ace_plan_config.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
    lib.ace_plan_tuning.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)]
    lib.ace_plan_radix.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(ctypes.c_float)]
    lib.ace_apply_prepare.argtypes = [P, ctypes.c_void_p, i32, ctypes.c_void_p]
    lib.ace_scdm.argtypes = [P, P, i32, i32, P, P, ctypes.POINTER(i32), P, P]
    lib.ace_apply_noalloc.argtypes = [P, i32, P, i32, i32, i32, P, P]
    lib.hfx_apply_exact.argtypes = [P, P, i32, f64, P, i32, P, P]
    lib.ace_last_intermediates.argtypes = [P, P, P, P]
    lib.ace_set_timing.argtypes = [P, i32]
    lib.ace_build_batched.argtypes = [ctypes.POINTER(_System), i32, P]
    lib.ace_save.argtypes = [ctypes.c_char_p, P, P, i32, f64, f64, P]
    lib.ace_load.argtypes = [ctypes.c_char_p, P, P, ctypes.POINTER(i32), ctypes.POINTER(f64), ctypes.POINTER(f64), P]
    lib.ace_get_stats.argtypes = [P, ctypes.POINTER(_Stats)]
    lib.ace_last_error.argtypes = [ctypes.c_char_p, i32]
    for name in SYMBOLS:
        if name != "ace_plan_destroy":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def last_error():
    """Message of this thread's last library error ("" if none)."""
    buf = ctypes.create_string_buffer(512)
    load().ace_last_error(buf, 512)
    return buf.value.decode()


def _check(code):
    if code != 0:
        raise AceError(code, last_error())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _plan_name(r0, n):
    """'r0 x n/r0' for a two-stage plan of an axis of length n (its first radix r0)."""
    if r0 <= 0:
        return None
    return f"{r0} x {n // r0}" if n // r0 > 1 else f"{r0}"


class Plan:
    """One system: grid, cell (rows = lattice vectors, bohr), cutoff (Ry),
    the largest occupied set, and the precision ("mixed" or "fp64").
    coulomb_rc = 0 solves Eq. 3 with 4 pi / |G|^2 and the G = 0 term dropped;
    coulomb_rc > 0 uses the interaction 1/r cut off at that radius (bohr;
    sphere_radius(cell) is the usual choice); coulomb_g0=True keeps the bare
    kernel's G = 0 term as the auxiliary-function (Gygi-Baldereschi) value."""

    def __init__(self, grid, cell, ecut, n_occ_max, precision="mixed", pair_batch=0, kernels=0, pair_streams=0,
                 pair_variant=0, coulomb_rc=0.0, coulomb_g0=False):
        lib = load()
        self.precision = precision
        self.prec = ACE_MIXED if precision == "mixed" else ACE_FP64
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.int32).reshape(3))
        c = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
        h = ctypes.c_void_p()
        opts = _Opts(int(pair_batch), int(kernels), int(pair_streams), int(pair_variant), float(coulomb_rc),
                     int(bool(coulomb_g0)))
        _check(lib.ace_plan_create(ctypes.byref(h), g.ctypes.data_as(ctypes.c_void_p),
                                   c.ctypes.data_as(ctypes.c_void_p), float(ecut), int(n_occ_max), self.prec,
                                   ctypes.byref(opts)))
        self.handle = h
        self.grid = tuple(int(x) for x in g)
        self.n_occ_max = int(n_occ_max)
        self.coulomb_rc = float(coulomb_rc)
        self.coulomb_g0 = bool(coulomb_g0)
        n = ctypes.c_int(0)
        _check(lib.ace_gvec(h, ctypes.byref(n), None))
        self.n_pw_half = n.value

    @property
    def cdtype(self):
        import torch
        return torch.complex64 if self.prec == ACE_MIXED else torch.complex128

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().ace_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def config(self):
        """dict(pair_variant, pair_streams, row_block, tune_ms, ...) of the pair-pass
        kernels (1 tile, 2 transposed planes, 3 persistent pipeline, 4 hybrid, 5 half-plane pairs)
        the pair-tile shape (ace_plan_tuning) and the pair passes' FFT radix plan
        (ace_plan_radix: first radix of every axis, and the candidates timed)."""
        v, st = ctypes.c_int(0), ctypes.c_int(0)
        tm = (ctypes.c_float * 6)()
        _check(load().ace_plan_config(self.handle, ctypes.byref(v), ctypes.byref(st), tm))
        rb, cached = ctypes.c_int(0), ctypes.c_int(0)
        rbm = (ctypes.c_float * 4)()
        _check(load().ace_plan_tuning(self.handle, ctypes.byref(rb), rbm, ctypes.byref(cached)))
        r0, nc = ctypes.c_int(0), ctypes.c_int(0)
        rc, rms = (ctypes.c_int * 4)(), (ctypes.c_float * 4)()
        _check(load().ace_plan_radix(self.handle, ctypes.byref(r0), ctypes.byref(nc), rc, rms))
        return {"pair_variant": v.value, "pair_streams": st.value, "row_block": rb.value,
                "radix_plan": _plan_name(r0.value, self.grid[0]),
                "radix_ms": {_plan_name(rc[k], self.grid[0]): round(float(rms[k]), 3)
                             for k in range(nc.value) if rms[k] > 0},
                "from_tune_cache": bool(cached.value),
                "tune_ms": {k: round(float(x), 3) for k, x in
                            zip(("tile_1_stream", "tile_2_streams", "planes", "pipeline", "hybrid", "half_planes"), tm)
                            if x > 0},
                "row_block_ms": {k: round(float(x), 3) for k, x in zip(("rows", "2", "4", "8"), rbm) if x > 0}}

    def _vec(self, t, name):
        if t.dtype != self.cdtype or not t.is_cuda or not t.is_contiguous() or t.dim() != 2 \
                or t.shape[1] != self.n_pw_half:
            raise ValueError(f"{name}: expected a contiguous CUDA {self.cdtype} tensor [rows][{self.n_pw_half}]")
        return t


def ace_plan_create(grid, cell, ecut, n_occ_max, precision="mixed", pair_batch=0, kernels=0, pair_streams=0,
                    pair_variant=0, coulomb_rc=0.0, coulomb_g0=False):
    """kernels: 0 fastest available, 1 CUDA-core Gram products, 2 also generic FFT passes;
    pair_streams: 0 automatic, 1 every pair pass in order on the call's stream;
    pair_variant: 0 automatic (timed at creation), 1 tile passes, 2 transposed planes,
    3 persistent pipeline, 4 hybrid (plane-kernel forward pass, tile passes after it);
    coulomb_rc: 0 bare Coulomb with G = 0 dropped, > 0 the interaction cut off at that radius;
    coulomb_g0: keep the bare kernel's G = 0 term as the auxiliary-function value."""
    return Plan(grid, cell, ecut, n_occ_max, precision, pair_batch, kernels, pair_streams, pair_variant, coulomb_rc,
                coulomb_g0)


def sphere_radius(cell):
    """(3 Omega / 4 pi)^(1/3) in bohr: the usual cutoff radius of the truncated
    Coulomb interaction (the sphere with the cell's volume)."""
    c = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    return float((3.0 * abs(np.linalg.det(c)) / (4.0 * np.pi)) ** (1.0 / 3.0))


def ace_plan_destroy(plan):
    plan.close()


def ace_gvec(plan):
    """Miller indices [n_pw_half, 3] of the plan's half sphere, canonical order."""
    m = np.zeros((plan.n_pw_half, 3), dtype=np.int32)
    n = ctypes.c_int(0)
    _check(load().ace_gvec(plan.handle, ctypes.byref(n), m.ctypes.data_as(ctypes.c_void_p)))
    return m


def ace_build(plan, psi_G, alpha, pairs=None, xi=None, stream=None):
    """Build the ACE vectors; returns (xi, E_x).  pairs = (row_ptr, col) CSR of
    kept pairs i <= j, or None for every pair."""
    import torch
    psi_G = plan._vec(psi_G, "psi_G")
    n_occ = psi_G.shape[0]
    if xi is None:
        xi = torch.empty_like(psi_G)
    plan._vec(xi, "xi")
    rp = col = None
    if pairs is not None:
        rp = np.ascontiguousarray(pairs[0], dtype=np.int32)
        col = np.ascontiguousarray(pairs[1], dtype=np.int32)
    E = ctypes.c_double(0.0)
    _check(load().ace_build(plan.handle, _ptr(psi_G), n_occ, float(alpha),
                            rp.ctypes.data_as(ctypes.c_void_p) if rp is not None else None,
                            col.ctypes.data_as(ctypes.c_void_p) if col is not None else None,
                            _ptr(xi), ctypes.byref(E), _stream(stream)))
    return xi, E.value


def ace_build_pairs(plan, psi_G, alpha, pairs=None, W_G=None, stream=None):
    """Pair half of a build split over shards: returns (W_G, E_part) over the
    listed pairs only.  pairs = (row_ptr, col) CSR over all n_occ rows (rows may
    be empty), or None for every pair."""
    import torch
    psi_G = plan._vec(psi_G, "psi_G")
    n_occ = psi_G.shape[0]
    if W_G is None:
        W_G = torch.empty_like(psi_G)
    plan._vec(W_G, "W_G")
    rp = col = None
    if pairs is not None:
        rp = np.ascontiguousarray(pairs[0], dtype=np.int32)
        col = np.ascontiguousarray(pairs[1], dtype=np.int32)
    E = ctypes.c_double(0.0)
    _check(load().ace_build_pairs(plan.handle, _ptr(psi_G), n_occ, float(alpha),
                                  rp.ctypes.data_as(ctypes.c_void_p) if rp is not None else None,
                                  col.ctypes.data_as(ctypes.c_void_p) if col is not None else None,
                                  _ptr(W_G), ctypes.byref(E), _stream(stream)))
    return W_G, E.value


def ace_build_async(plan, psi_G, alpha, pairs=None, xi=None, stream=None):
    """Enqueue a build without host synchronisation (CUDA-graph capturable once
    the same call has run outside capture); returns xi.  Read E_x with
    ace_build_result after the stream completes.  The pair arrays are kept
    on the plan object until the next enqueue."""
    import torch
    psi_G = plan._vec(psi_G, "psi_G")
    n_occ = psi_G.shape[0]
    if xi is None:
        xi = torch.empty_like(psi_G)
    plan._vec(xi, "xi")
    rp = col = None
    if pairs is not None:
        rp = np.ascontiguousarray(pairs[0], dtype=np.int32)
        col = np.ascontiguousarray(pairs[1], dtype=np.int32)
    plan._async_pairs = (rp, col)
    _check(load().ace_build_async(plan.handle, _ptr(psi_G), n_occ, float(alpha),
                                  rp.ctypes.data_as(ctypes.c_void_p) if rp is not None else None,
                                  col.ctypes.data_as(ctypes.c_void_p) if col is not None else None,
                                  _ptr(xi), _stream(stream)))
    return xi


def ace_check_timeout_path(plan, limit_ms=50, stream=None):
    """Run the bounded-wait failure path once (a wait nothing completes);
    returns the status code (ACE_ERR_TIMEOUT expected) without raising."""
    return int(load().ace_check_timeout_path(plan.handle, int(limit_ms), _stream(stream)))


def ace_build_result(plan, stream=None):
    """E_x of the last ace_build_async (waits for the stream)."""
    E = ctypes.c_double(0.0)
    _check(load().ace_build_result(plan.handle, ctypes.byref(E), _stream(stream)))
    return E.value


def ace_scdm(plan, psi_G, preselect=True, phi_G=None, stream=None):
    """SCDM localisation (Section 2.4) with the s'-MTACE pre-selection
    (Section 2.5, preselect=True): returns (phi_G, pivots, O, n_candidates) --
    the localised orbitals (same layout and precision as psi_G), the pivot grid
    points (i0 n1 + i1) n2 + i2, the orthogonal rotation phi = O psi (float64
    numpy) and how many grid points were candidates."""
    import torch

    psi_G = plan._vec(psi_G, "psi_G")
    n = psi_G.shape[0]
    if phi_G is None:
        phi_G = torch.empty_like(psi_G)
    else:
        phi_G = plan._vec(phi_G, "phi_G")
    piv = np.zeros(n, dtype=np.int32)
    O = np.zeros((n, n), dtype=np.float64)
    nc = ctypes.c_int(0)
    _check(load().ace_scdm(plan.handle, _ptr(psi_G), n, int(bool(preselect)), _ptr(phi_G),
                           piv.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nc), O.ctypes.data_as(ctypes.c_void_p),
                           _stream(stream)))
    return phi_G, piv, O, nc.value


def ace_overlap_screen(plan, psi_G, rho_cut, stream=None):
    """s-MTACE screening (Section 2.4): returns (pairs, S) with pairs = (row_ptr,
    col) of the i <= j kept by S_ij = int |phi_i phi_j| >= rho_cut (diagonal
    always) and S the [n_occ][n_occ] overlaps (float64 numpy)."""
    psi_G = plan._vec(psi_G, "psi_G")
    n = psi_G.shape[0]
    rp = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(max(1, n * (n + 1) // 2), dtype=np.int32)
    S = np.zeros((n, n), dtype=np.float64)
    npairs = ctypes.c_int(0)
    _check(load().ace_overlap_screen(plan.handle, _ptr(psi_G), n, float(rho_cut), rp.ctypes.data_as(ctypes.c_void_p),
                                     col.ctypes.data_as(ctypes.c_void_p), ctypes.byref(npairs),
                                     S.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return (rp, col[:npairs.value].copy()), S


def ace_build_finish(plan, psi_G, W_G, xi=None, stream=None):
    """Dense half of a split build: M = Phi^T W, Cholesky, xi = W L^-T, from
    W_G summed over the shards."""
    import torch
    psi_G = plan._vec(psi_G, "psi_G")
    plan._vec(W_G, "W_G")
    if xi is None:
        xi = torch.empty_like(psi_G)
    plan._vec(xi, "xi")
    _check(load().ace_build_finish(plan.handle, _ptr(psi_G), psi_G.shape[0], _ptr(W_G), _ptr(xi),
                                   _stream(stream)))
    return xi


def ace_apply(plan, xi, psi, out=None, stream=None):
    """K psi = -xi (xi^T psi)."""
    import torch
    plan._vec(xi, "xi")
    plan._vec(psi, "psi")
    if out is None:
        out = torch.empty_like(psi)
    plan._vec(out, "out")
    _check(load().ace_apply(plan.handle, _ptr(xi), xi.shape[0], _ptr(psi), psi.shape[0], _ptr(out),
                            _stream(stream)))
    return out


def ace_apply_prepare(plan, xi, stream=None):
    """Make the plan's split copy of xi for the inner steps that follow
    (ace_apply_prepare): later ace_apply calls with this xi read it until the
    next build, load or prepare on the plan."""
    plan._vec(xi, "xi")
    _check(load().ace_apply_prepare(plan.handle, _ptr(xi), xi.shape[0], _stream(stream)))


def ace_apply_energy(plan, xi, psi, stream=None):
    """sum_t <psi_t|K psi_t> = -sum_{t,k} <xi_k|psi_t>^2 (the fast energy of an
    inner MTS step), reduced on the device; returns a float."""
    plan._vec(xi, "xi")
    plan._vec(psi, "psi")
    E = ctypes.c_double(0.0)
    _check(load().ace_apply_energy(plan.handle, _ptr(xi), xi.shape[0], _ptr(psi), psi.shape[0], ctypes.byref(E),
                                   _stream(stream)))
    return E.value


def hfx_apply_exact(plan, psi_occ, alpha, psi, out=None, stream=None):
    """alpha V_X psi with the exact exchange operator of the occupied set."""
    import torch
    plan._vec(psi_occ, "psi_occ")
    plan._vec(psi, "psi")
    if out is None:
        out = torch.empty_like(psi)
    plan._vec(out, "out")
    _check(load().hfx_apply_exact(plan.handle, _ptr(psi_occ), psi_occ.shape[0], float(alpha), _ptr(psi),
                                  psi.shape[0], _ptr(out), _stream(stream)))
    return out


def ace_last_intermediates(plan, n_occ, stream=None):
    """(W_G, M) of the last ace_build: W_G on the device, M as a numpy array."""
    import torch
    W = torch.empty((n_occ, plan.n_pw_half), dtype=plan.cdtype, device="cuda")
    M = np.zeros((n_occ, n_occ))
    _check(load().ace_last_intermediates(plan.handle, _ptr(W), M.ctypes.data_as(ctypes.c_void_p),
                                         _stream(stream)))
    return W, M


def ace_set_timing(plan, enable=True):
    """Record CUDA events at phase boundaries of the following calls."""
    _check(load().ace_set_timing(plan.handle, 1 if enable else 0))


def ace_get_stats(plan):
    """Per-phase device milliseconds and counters since the last call (resets them)."""
    st = _Stats()
    _check(load().ace_get_stats(plan.handle, ctypes.byref(st)))
    d = {f: getattr(st, f) for f in STAT_FIELDS}
    d["pair_transforms"] = st.pair_transforms
    d["launches"] = st.launches
    d["pair_wall_ms"] = st.pair_wall_ms
    return d


def ace_apply_noalloc(xi, psi, out, stream=None):
    """K psi = -xi (xi^T psi) without a plan and without device allocation in
    the library (for callers that must not allocate).  xi, psi and out are
    caller-owned contiguous CUDA tensors: complex64 (mixed) or complex128
    (fp64) of shape [rows][n_pw_half], all on the current CUDA device;
    T * n_occ <= 524288.  Raises ValueError before the library is called
    when a tensor has another dtype, layout or device."""
    import torch
    if xi.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("ace_apply_noalloc: xi must be complex64 (mixed) or complex128 (fp64)")
    prec = ACE_MIXED if xi.dtype == torch.complex64 else ACE_FP64
    for t in (xi, psi, out):
        if not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or t.dtype != xi.dtype or t.shape[1] != xi.shape[1]:
            raise ValueError("ace_apply_noalloc: contiguous CUDA complex tensors of one dtype and width")
    here = torch.device("cuda", torch.cuda.current_device())
    if any(t.device != here for t in (xi, psi, out)):
        raise ValueError(f"ace_apply_noalloc: xi, psi and out must be on the current device {here}")
    if out.shape != psi.shape:
        raise ValueError("ace_apply_noalloc: out must have the shape of psi")
    _check(load().ace_apply_noalloc(_ptr(xi), xi.shape[0], _ptr(psi), psi.shape[0], xi.shape[1], prec, _ptr(out),
                                    _stream(stream)))
    return out


def ace_build_batched(systems, stream=None):
    """Build several independent systems in one call.  systems: list of dicts
    with plan, psi_G, alpha and optionally pairs (row_ptr, col).  Returns a list
    of (xi, E_x); raises on the first failing system."""
    import torch
    arr = (_System * len(systems))()
    keep = []
    outs = []
    for k, s in enumerate(systems):
        plan = s["plan"]
        psi = plan._vec(s["psi_G"], "psi_G")
        xi = torch.empty_like(psi)
        rp = col = None
        if s.get("pairs") is not None:
            rp = np.ascontiguousarray(s["pairs"][0], dtype=np.int32)
            col = np.ascontiguousarray(s["pairs"][1], dtype=np.int32)
            keep += [rp, col]
        arr[k] = _System(plan.handle.value, psi.data_ptr(), psi.shape[0], float(s["alpha"]),
                         rp.ctypes.data if rp is not None else None, col.ctypes.data if col is not None else None,
                         xi.data_ptr(), 0.0, 0)
        outs.append(xi)
    _check(load().ace_build_batched(arr, len(systems), _stream(stream)))
    return [(outs[k], arr[k].E_x) for k in range(len(systems))]


class BatchedBuildGraph:
    """Several independent systems (each with its own plan) built by one CUDA
    graph launch: every system's ace_build_async captured on its own stream,
    forked from and joined back into the capturing stream, after one run of
    the same calls outside capture (allocations, attributes).  replay() runs
    all the builds and returns their E_x; each system's xi is filled in place.
    systems: list of dicts with plan, psi_G (captured by address: copy new
    orbitals into it before a replay), alpha and optionally pairs."""

    def __init__(self, systems):
        import torch
        self.systems = systems
        self.xi = [torch.empty_like(s["psi_G"]) for s in systems]
        for s, xi in zip(systems, self.xi):
            ace_build_async(s["plan"], s["psi_G"], s["alpha"], pairs=s.get("pairs"), xi=xi)
        for s in systems:
            ace_build_result(s["plan"])
        self.streams = [torch.cuda.Stream() for _ in systems]
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            main = torch.cuda.current_stream()
            for s, xi, side in zip(systems, self.xi, self.streams):
                side.wait_stream(main)
                with torch.cuda.stream(side):
                    ace_build_async(s["plan"], s["psi_G"], s["alpha"], pairs=s.get("pairs"), xi=xi, stream=side)
            for side in self.streams:
                main.wait_stream(side)

    def launch(self):
        """Replay the graph without waiting for it."""
        self.graph.replay()

    def replay(self):
        """Replay and return every system's E_x (waits for the graph)."""
        import torch
        self.graph.replay()
        torch.cuda.current_stream().synchronize()
        return [ace_build_result(s["plan"]) for s in self.systems]


def ace_save(plan, path, xi, alpha, E_x, stream=None):
    plan._vec(xi, "xi")
    _check(load().ace_save(os.fsencode(path), plan.handle, _ptr(xi), xi.shape[0], float(alpha), float(E_x),
                           _stream(stream)))


def ace_load(plan, path, stream=None):
    """(xi, alpha, E_x) saved by ace_save for a plan of the same geometry."""
    import torch
    buf = torch.empty((plan.n_occ_max, plan.n_pw_half), dtype=plan.cdtype, device="cuda")
    n = ctypes.c_int(0)
    a = ctypes.c_double(0)
    e = ctypes.c_double(0)
    _check(load().ace_load(os.fsencode(path), plan.handle, _ptr(buf), ctypes.byref(n), ctypes.byref(a),
                           ctypes.byref(e), _stream(stream)))
    return buf[:n.value].clone(), a.value, e.value
