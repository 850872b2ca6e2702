"""Thin ctypes binding of libimex (include/imex.h): argument marshalling only.

Every step of the time integration runs in the library's CUDA kernels; this
module converts Python/NumPy/PyTorch arguments to the C structs, passes device
pointers and streams through, and raises on error codes.  If libimex.so is
missing it raises ImportError: there is no Python or CPU fallback.

PyTorch supplies device memory (through the allocator hooks) and streams.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libimex.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libimex.so not built ({LIB_PATH}); run "
                      "`python -m paper_2310_14712_gb300.build` (needs nvcc)")

_lib = ctypes.CDLL(LIB_PATH)

OK = 0
ERR = {-1: "IMEX_ERR_ARG", -2: "IMEX_ERR_GEOM", -3: "IMEX_ERR_ALLOC", -4: "IMEX_ERR_CUDA",
       -5: "IMEX_ERR_NOT_SPD", -6: "IMEX_ERR_TIMEOUT", -7: "IMEX_ERR_DIVERGED"}

FIELD_U, FIELD_U_PREV_D, FIELD_V_C, FIELD_A_C, FIELD_FX, FIELD_MASK_D, FIELD_MASK_C = range(7)
FIELDS = {"u": FIELD_U, "u_prev_d": FIELD_U_PREV_D, "v_c": FIELD_V_C, "a_c": FIELD_A_C,
          "fx": FIELD_FX, "mask_d": FIELD_MASK_D, "mask_c": FIELD_MASK_C}

_dp = ctypes.POINTER(ctypes.c_double)


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("ncells", ctypes.c_int * 3), ("nholes", ctypes.c_int), ("holes", _dp),
                ("tree_depth", ctypes.c_int), ("rho", ctypes.c_double), ("c0", ctypes.c_double),
                ("cell_c", _dp)]


class Source(ctypes.Structure):
    _fields_ = [("nsrc", ctypes.c_int), ("pos", _dp), ("f0", ctypes.c_double),
                ("sigma", ctypes.c_double), ("amp", ctypes.c_double), ("wavelet", ctypes.c_int)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Alloc(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("user", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_nodes", "n_d", "n_c", "n_cut", "n_uncut", "n_empty", "n_iface", "nnz_L",
        "n_components", "n_tree", "max_block", "step", "device_bytes")] + \
        [(n, ctypes.c_double) for n in ("dt", "dt_crit_uncut", "setup_seconds", "residual_S", "residual_M")] + \
        [(n, ctypes.c_int64) for n in ("solve_levels", "solve_ctas", "solve_smem_bytes", "launches_per_step",
                                    "rhs_pairs", "ncols", "explicit_tile_cells")] + \
        [(n, ctypes.c_double) for n in ("explicit_tile_us_large", "explicit_tile_us_small")] + \
        [("scheme", ctypes.c_int64), ("dt_crit_cut_min", ctypes.c_double), ("factorized", ctypes.c_int64),
         ("explicit_variant", ctypes.c_int64), ("explicit_sweep_us", ctypes.c_double),
         ("explicit_sweep_short_us", ctypes.c_double), ("large_supernodes", ctypes.c_int64),
         ("max_rows", ctypes.c_int64), ("solve_smem_needed", ctypes.c_int64),
         ("explicit_split_us", ctypes.c_double * 4), ("solve_col_block", ctypes.c_int64),
         ("solve_col_block_us", ctypes.c_double * 7)]

    def as_dict(self):
        out = {n: getattr(self, n) for n, _ in self._fields_}
        out["explicit_split_us"] = list(out["explicit_split_us"])
        out["solve_col_block_us"] = list(out["solve_col_block_us"])
        return out


_vp = ctypes.c_void_p
_lib.imex_setup.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                            ctypes.POINTER(Source), ctypes.POINTER(Alloc), ctypes.POINTER(_vp)]
_lib.imex_setup_batch.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(Source), ctypes.c_int, ctypes.POINTER(Alloc),
                                  ctypes.POINTER(_vp)]
_lib.imex_setup_scheme.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(Source), ctypes.c_int, ctypes.c_int, ctypes.POINTER(Alloc),
                                   ctypes.POINTER(_vp)]
_lib.imex_setup_pcg.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(Source), ctypes.c_int, ctypes.POINTER(Alloc), ctypes.POINTER(_vp)]
_lib.imex_step.argtypes = [_vp, ctypes.c_int64, _vp]
_lib.imex_check_finite.argtypes = [_vp, _dp]
_lib.imex_adjoint.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, _dp,
                              ctypes.c_int, _dp, _dp]
_lib.imex_set_solver.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]
_lib.imex_pcg_train.argtypes = [_vp, ctypes.c_int, ctypes.c_double, _dp]
_lib.imex_pcg_train_guess.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
_lib.imex_pcg_set_guess.argtypes = [_vp, ctypes.c_int, _dp]
_lib.imex_pcg_fsai_closed_form.argtypes = [_vp]
_lib.imex_pcg_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), _dp, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64)]
_lib.imex_fsai_kaporin.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _dp, _vp]
_lib.imex_step_profile.argtypes = [_vp, ctypes.c_int64, _vp, _dp]
_lib.imex_step_io.argtypes = [_vp, ctypes.c_int64, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                              _dp, _vp]
_lib.imex_step_noalloc.argtypes = [_vp, ctypes.c_int64, _vp]
_lib.imex_fields.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int64, ctypes.c_int]
_lib.imex_set_fields.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int64, ctypes.c_int]
_lib.imex_set_step.argtypes = [_vp, ctypes.c_int64]
_lib.imex_set_initial.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int]
_lib.imex_info.argtypes = [_vp, ctypes.POINTER(Stats)]
_lib.imex_probe_fp64.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
_lib.imex_last_error.restype = ctypes.c_char_p
_lib.imex_destroy.argtypes = [_vp]
_lib.imex_destroy.restype = None
_lib.imex_gll_points.argtypes = [ctypes.c_int, _dp, _dp]
_lib.imex_gauss_points.argtypes = [ctypes.c_int, _dp, _dp]
_lib.imex_host_setup_export.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(Source), _vp, _dp,
                                        ctypes.POINTER(Stats)]
_lib.imex_host_element_matrices.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double,
                                            ctypes.POINTER(Source), ctypes.c_int, _vp, _dp, _dp, _vp]
_lib.imex_host_implicit_system.argtypes = [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(Source), _vp, _vp, _vp, _vp, _vp, _dp, _dp]

# Every symbol include/imex.h declares (checked by the CPU tests).
EXPORTS = ("imex_setup", "imex_setup_batch", "imex_setup_scheme", "imex_setup_pcg", "imex_adjoint", "imex_set_solver", "imex_pcg_train", "imex_pcg_train_guess", "imex_pcg_set_guess", "imex_pcg_fsai_closed_form", "imex_pcg_status",
           "imex_fsai_kaporin", "imex_step", "imex_step_profile", "imex_step_io", "imex_step_noalloc", "imex_fields", "imex_set_fields", "imex_set_step",
           "imex_set_initial", "imex_info", "imex_check_finite", "imex_last_error", "imex_destroy", "imex_gll_points",
           "imex_gauss_points", "imex_host_setup_export", "imex_host_element_matrices", "imex_host_implicit_system",
           "imex_probe_fp64")


class ImexError(RuntimeError):
    def __init__(self, code, what):
        msg = _lib.imex_last_error().decode()
        super().__init__(f"{what}: {ERR.get(code, code)}: {msg}")
        self.code = code


def _check(code, what):
    if code != OK:
        raise ImexError(code, what)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _mesh_source(dim, lo, hi, ncells, depth, holes, rho, c0, cell_c, src_pos, f0, sigma, amp, wavelet):
    keep = []
    m = Mesh()
    m.dim = dim
    for k in range(3):
        m.lo[k] = lo[k] if k < dim else 0.0
        m.hi[k] = hi[k] if k < dim else 1.0
        m.ncells[k] = ncells[k] if k < dim else 1
    h = _f64(holes).reshape(-1)
    keep.append(h)
    m.nholes = len(h) // (2 * dim)
    m.holes = h.ctypes.data_as(_dp) if len(h) else None
    m.tree_depth = depth
    m.rho = rho
    m.c0 = c0
    if cell_c is not None:
        cc = _f64(cell_c).reshape(-1)
        keep.append(cc)
        m.cell_c = cc.ctypes.data_as(_dp)
    else:
        m.cell_c = None
    s = Source()
    pos = _f64(src_pos).reshape(-1)
    keep.append(pos)
    s.nsrc = len(pos) // dim
    s.pos = pos.ctypes.data_as(_dp)
    s.f0, s.sigma, s.amp, s.wavelet = f0, sigma, amp, wavelet
    return m, s, keep


SOLVERS = {"direct": 0, "pcg_fsai": 1, "pcg_jacobi": 2}
# Time integration schemes (IMEX_SCHEME_*): the method and the paper's comparison schemes.
SCHEMES = {"imex": 0, "cdm": 1, "cdm_hrz": 2, "trapezoidal": 3}


def fsai_kaporin(s_ptr, s_col, s_val, g_ptr, g_col, g_val, stream=None):
    """K(G) = tr(G^T S G) - 2 sum log G_ii and its gradient with the library's
    training kernels; all arguments are CUDA torch tensors (int32 / float64,
    CSR).  Returns (loss, grad tensor)."""
    import torch
    n = int(s_ptr.numel()) - 1
    grad = torch.empty_like(g_val)
    loss = ctypes.c_double(0.0)
    st = torch.cuda.current_stream() if stream is None else stream
    _check(_lib.imex_fsai_kaporin(n, s_ptr.data_ptr(), s_col.data_ptr(), s_val.data_ptr(), g_ptr.data_ptr(),
                                  g_col.data_ptr(), g_val.data_ptr(), grad.data_ptr(), ctypes.byref(loss),
                                  ctypes.c_void_p(st.cuda_stream)), "imex_fsai_kaporin")
    return loss.value, grad


PROBE_KINDS = {"fma": 0, "add": 1, "mul": 2}


def probe_fp64(kind="fma", iters=40000):
    """Measured FP64 thread-instruction rate of the current device (imex_probe_fp64):
    returns (instructions per second, seconds of the timed launch)."""
    rate, secs = ctypes.c_double(), ctypes.c_double()
    _check(_lib.imex_probe_fp64(PROBE_KINDS[kind], int(iters), ctypes.byref(rate), ctypes.byref(secs)),
           "imex_probe_fp64")
    return rate.value, secs.value


def gll_points(p):
    x = np.zeros(p + 1)
    w = np.zeros(p + 1)
    _check(_lib.imex_gll_points(p, x.ctypes.data_as(_dp), w.ctypes.data_as(_dp)), "imex_gll_points")
    return x, w


def gauss_points(n):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(_lib.imex_gauss_points(n, x.ctypes.data_as(_dp), w.ctypes.data_as(_dp)), "imex_gauss_points")
    return x, w


def host_setup_export(dim, lo, hi, ncells, p, alpha, depth, holes, src_pos, f0, src_sigma,
                      src_amp=10.0, wavelet=0, rho=1.0, c0=1.0, cell_c=None, dt=0.0, **_):
    """Host setup only (no GPU): node classes, f_x and counts."""
    m, s, keep = _mesh_source(dim, lo, hi, ncells, depth, holes, rho, c0, cell_c, src_pos, f0,
                              src_sigma, src_amp, wavelet)
    nn = int(np.prod([ncells[k] * p + 1 for k in range(dim)]))
    cls = np.zeros(nn, dtype=np.uint8)
    fx = np.zeros(nn)
    st = Stats()
    _check(_lib.imex_host_setup_export(ctypes.byref(m), p, alpha, dt, ctypes.byref(s),
                                       cls.ctypes.data, fx.ctypes.data_as(_dp), ctypes.byref(st)),
           "imex_host_setup_export")
    return cls, fx, st.as_dict()


def host_element_matrices(cells, dim, lo, hi, ncells, p, alpha, depth, holes, src_pos, f0, src_sigma,
                          src_amp=10.0, wavelet=0, rho=1.0, c0=1.0, cell_c=None, **_):
    """Host discretisation only (no GPU): element matrices K_e, M_e of the
    given flat cell ids as the library assembles them, shape (n, P^d, P^d),
    and the cell types (0 uncut, 1 cut, 2 empty)."""
    m, s, keep = _mesh_source(dim, lo, hi, ncells, depth, holes, rho, c0, cell_c, src_pos, f0,
                              src_sigma, src_amp, wavelet)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    Pd = (p + 1) ** dim
    K = np.zeros((len(cells), Pd, Pd))
    M = np.zeros((len(cells), Pd, Pd))
    types = np.zeros(len(cells), dtype=np.int8)
    _check(_lib.imex_host_element_matrices(ctypes.byref(m), p, alpha, ctypes.byref(s), len(cells),
                                           cells.ctypes.data, K.ctypes.data_as(_dp), M.ctypes.data_as(_dp),
                                           types.ctypes.data), "imex_host_element_matrices")
    # column-major per cell -> (row, column)
    return K.transpose(0, 2, 1).copy(), M.transpose(0, 2, 1).copy(), types


def host_implicit_system(dim, lo, hi, ncells, p, alpha, depth, holes, src_pos, f0, src_sigma,
                         src_amp=10.0, wavelet=0, rho=1.0, c0=1.0, cell_c=None, dt=0.0, **_):
    """Host setup only (no GPU): the implicit system S = M^cc + dt^2/4 K^cc
    and M^cc as the library factorises them, as (c_node, s_ptr, s_col, s_val,
    m_val) in the library's c-order (CSR)."""
    m, s, keep = _mesh_source(dim, lo, hi, ncells, depth, holes, rho, c0, cell_c, src_pos, f0,
                              src_sigma, src_amp, wavelet)
    n_c = ctypes.c_int64(0)
    nnz = ctypes.c_int64(0)
    _check(_lib.imex_host_implicit_system(ctypes.byref(m), p, alpha, dt, ctypes.byref(s), ctypes.byref(n_c),
                                          ctypes.byref(nnz), None, None, None, None, None),
           "imex_host_implicit_system")
    c_node = np.zeros(n_c.value, dtype=np.int64)
    ptr = np.zeros(n_c.value + 1, dtype=np.int64)
    col = np.zeros(nnz.value, dtype=np.int32)
    sv = np.zeros(nnz.value)
    mv = np.zeros(nnz.value)
    _check(_lib.imex_host_implicit_system(ctypes.byref(m), p, alpha, dt, ctypes.byref(s), ctypes.byref(n_c),
                                          ctypes.byref(nnz), c_node.ctypes.data, ptr.ctypes.data, col.ctypes.data,
                                          sv.ctypes.data_as(_dp), mv.ctypes.data_as(_dp)),
           "imex_host_implicit_system")
    return c_node, ptr, col, sv, mv


class _TorchAllocator:
    """Device allocations served by PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.blocks = {}
        self._alloc = _ALLOC_FN(self._do_alloc)
        self._release = _RELEASE_FN(self._do_release)
        self.struct = Alloc(self._alloc, self._release, None)

    def _do_alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        self.blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _do_release(self, ptr, user):
        self.blocks.pop(ptr, None)


class Imex:
    """One immersed Newmark IMEX problem on the current CUDA device.

    Construct from a workload (paper_2310_14712_gb300.workloads.Workload) or
    from explicit arguments.  Device memory comes from PyTorch.  With
    ncols > 1 the context steps ncols independent simulations, column k
    loaded by the source at src_pos[k] alone (imex_setup_batch); fields then
    have ncols * n_nodes entries, column after column.  `scheme` picks the
    time integration (SCHEMES; imex_setup_scheme): the method itself or one of
    the paper's comparison schemes on the same discretisation.  With
    factorize=False the implicit solve is PCG only (imex_setup_pcg).
    """

    def __init__(self, dim, lo, hi, ncells, p, alpha, depth, holes, src_pos, f0, src_sigma,
                 src_amp=10.0, wavelet=0, rho=1.0, c0=1.0, cell_c=None, dt=0.0, use_torch_alloc=True,
                 ncols=1, scheme="imex", factorize=True, **_):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device("cuda", torch.cuda.current_device())
        m, s, keep = _mesh_source(dim, lo, hi, ncells, depth, holes, rho, c0, cell_c, src_pos, f0,
                                  src_sigma, src_amp, wavelet)
        self._allocator = _TorchAllocator(self.device) if use_torch_alloc else None
        ctx = _vp()
        al = ctypes.byref(self._allocator.struct) if self._allocator else None
        if factorize:
            _check(_lib.imex_setup_scheme(ctypes.byref(m), p, alpha, dt, ctypes.byref(s), int(ncols),
                                          SCHEMES[scheme], al, ctypes.byref(ctx)), "imex_setup_scheme")
        else:   # no factorisation: PCG only (imex_setup_pcg), one column
            if int(ncols) != 1:
                raise ValueError("a context without a factorisation has one column")
            _check(_lib.imex_setup_pcg(ctypes.byref(m), p, alpha, dt, ctypes.byref(s), SCHEMES[scheme], al,
                                       ctypes.byref(ctx)), "imex_setup_pcg")
        self._ctx = ctx
        self.stats = self.info()
        self.n_nodes = self.stats["n_nodes"]
        self.ncols = int(ncols)
        self.field_len = self.n_nodes * self.ncols
        self.dim = dim
        self.shape = tuple(reversed([ncells[k] * p + 1 for k in range(dim)]))
        self._ncells = tuple(ncells[:dim])

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(**w.kwargs(), **kw)

    def _stream(self, stream):
        if stream is None:
            stream = self.torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(stream.cuda_stream)

    def step(self, n, stream=None):
        """Advance n IMEX steps asynchronously on `stream` (default: torch's current stream)."""
        _check(_lib.imex_step(self._ctx, int(n), self._stream(stream)), "imex_step")

    def set_solver(self, solver="direct", tol=1e-10, maxit=200):
        """'direct' (factorised), 'pcg_fsai' (learned G G^T) or 'pcg_jacobi'."""
        _check(_lib.imex_set_solver(self._ctx, SOLVERS[solver], float(tol), int(maxit)), "imex_set_solver")

    def pcg_train(self, epochs, lr=3e-2):
        """Adam steps on Kaporin's functional for G; returns the loss before each step."""
        hist = np.zeros(int(epochs))
        _check(_lib.imex_pcg_train(self._ctx, int(epochs), float(lr), hist.ctypes.data_as(_dp)), "imex_pcg_train")
        return hist

    def adjoint(self, nsteps, rec_nodes, data, checkpoint_every=100):
        """Misfit of the next nsteps steps at the receivers against data
        (nsteps x ncols x nrec) and its gradient in the per-cell wave speed."""
        rec = np.ascontiguousarray(np.asarray(rec_nodes, dtype=np.int64))
        d = _f64(data).reshape(int(nsteps), self.ncols, len(rec))
        ncell = int(np.prod(self._ncells))
        grad = np.zeros(ncell)
        J = ctypes.c_double()
        _check(_lib.imex_adjoint(self._ctx, int(nsteps), rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 len(rec), d.ctypes.data_as(_dp), int(checkpoint_every),
                                 grad.ctypes.data_as(_dp), ctypes.byref(J)), "imex_adjoint")
        return J.value, grad

    def pcg_train_guess(self, nsteps, epochs, lr=0.05):
        """Advance nsteps steps, then learn the PCG starting-guess weights from
        their solutions (imex_pcg_train_guess); returns (weights, loss history)."""
        hist = np.zeros(max(int(epochs), 1))
        w = np.zeros(3)
        _check(_lib.imex_pcg_train_guess(self._ctx, int(nsteps), int(epochs), float(lr), hist.ctypes.data_as(_dp),
                                         w.ctypes.data_as(_dp)), "imex_pcg_train_guess")
        return w, hist[:int(epochs)]

    def pcg_set_guess(self, enable=True, w=None):
        """Enable (given or trained weights) or disable the learned PCG starting guess."""
        wp = None
        if w is not None:
            w = _f64(w)
            wp = w.ctypes.data_as(_dp)
        _check(_lib.imex_pcg_set_guess(self._ctx, 1 if enable else 0, wp), "imex_pcg_set_guess")

    def pcg_fsai_closed_form(self):
        """Set G to the closed-form FSAI of its pattern (imex_pcg_fsai_closed_form)."""
        _check(_lib.imex_pcg_fsai_closed_form(self._ctx), "imex_pcg_fsai_closed_form")

    def pcg_status(self):
        it, tot, fb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        res = ctypes.c_double()
        _check(_lib.imex_pcg_status(self._ctx, ctypes.byref(it), ctypes.byref(res), ctypes.byref(tot),
                                    ctypes.byref(fb)), "imex_pcg_status")
        return {"iters_last": it.value, "res_last": res.value, "iters_total": tot.value, "fallbacks": fb.value}

    def step_noalloc(self, n, stream=None):
        """Like step(), but the implicit solve's scratch lives in the library's fixed
        2 MiB device array and the call allocates nothing (see include/imex.h)."""
        _check(_lib.imex_step_noalloc(self._ctx, int(n), self._stream(stream)), "imex_step_noalloc")

    PROFILE_PHASES = ("explicit", "implicit", "step")

    def step_profile(self, n, stream=None):
        """Advance n steps with CUDA events around the kernels; returns the summed
        device ms of (explicit + CDM + prediction, implicit chain: right-hand sides,
        solve and correction, whole steps), in PROFILE_PHASES order."""
        ms = (ctypes.c_double * len(self.PROFILE_PHASES))()
        _check(_lib.imex_step_profile(self._ctx, int(n), self._stream(stream), ms), "imex_step_profile")
        return tuple(ms)

    def step_io(self, n, ft_samples, rec_nodes, traces, stream=None):
        """n steps with host I/O every step: ft_samples (n+1 host doubles, or None for
        the built-in wavelet), receivers rec_nodes (int64 node ids); traces (n x ncols x
        nrec host doubles) receives u at the receivers after every step.  Host arrays may
        be pinned torch CPU tensors or NumPy arrays."""
        def ptr(a, ct):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                return a.ctypes.data_as(ctypes.POINTER(ct))
            return ctypes.cast(a.data_ptr(), ctypes.POINTER(ct))
        nrec = len(rec_nodes)
        _check(_lib.imex_step_io(self._ctx, int(n), ptr(ft_samples, ctypes.c_double),
                                 ptr(rec_nodes, ctypes.c_int64), nrec, ptr(traces, ctypes.c_double),
                                 self._stream(stream)), "imex_step_io")

    def fields(self, which="u", out=None):
        """Copy a field (canonical layout; ncols grids one after the other) into `out`
        (torch CUDA tensor or NumPy array)."""
        code = FIELDS[which] if isinstance(which, str) else int(which)
        n = self.field_len
        if out is None:
            out = self.torch.empty(n, dtype=self.torch.float64, device=self.device)
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float64 and out.size == n and out.flags.c_contiguous
            _check(_lib.imex_fields(self._ctx, code, out.ctypes.data, n, 0), "imex_fields")
        else:
            assert out.dtype == self.torch.float64 and out.numel() == n and out.is_contiguous()
            _check(_lib.imex_fields(self._ctx, code, out.data_ptr(), n, 1 if out.is_cuda else 0),
                   "imex_fields")
        return out

    def set_fields(self, which, src):
        code = FIELDS[which] if isinstance(which, str) else int(which)
        n = self.field_len
        if isinstance(src, np.ndarray):
            src = _f64(src)
            _check(_lib.imex_set_fields(self._ctx, code, src.ctypes.data, n, 0), "imex_set_fields")
        else:
            src = src.contiguous()
            _check(_lib.imex_set_fields(self._ctx, code, src.data_ptr(), n, 1 if src.is_cuda else 0),
                   "imex_set_fields")

    def set_step(self, n):
        _check(_lib.imex_set_step(self._ctx, int(n)), "imex_set_step")

    def set_initial(self, u0, v0=None):
        u0 = _f64(u0)
        v0p = None
        if v0 is not None:
            v0 = _f64(v0)
            v0p = v0.ctypes.data
        _check(_lib.imex_set_initial(self._ctx, u0.ctypes.data, v0p, self.field_len, 0), "imex_set_initial")

    def check_finite(self):
        """max |u_n| over the active DOFs; raises ImexError (IMEX_ERR_DIVERGED) if
        the state holds a non-finite value."""
        m = ctypes.c_double()
        _check(_lib.imex_check_finite(self._ctx, ctypes.byref(m)), "imex_check_finite")
        return m.value

    def info(self):
        st = Stats()
        _check(_lib.imex_info(self._ctx, ctypes.byref(st)), "imex_info")
        return st.as_dict()

    def close(self):
        if getattr(self, "_ctx", None):
            _lib.imex_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
