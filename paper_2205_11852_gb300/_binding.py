"""ctypes binding of libtpcf (include/tpcf.h): argument marshalling only.

Every computation runs in the CUDA library; this module builds the C
structs, passes device pointers of torch CUDA tensors (torch supplies the
device memory and the current stream) and turns return codes into
exceptions.  There is no CPU fallback: if ``_build/libtpcf.so`` is missing
the import fails.
"""
from __future__ import annotations

import ctypes
import math
import pathlib

import torch

_LIBPATH = pathlib.Path(__file__).resolve().parent / "_build" / "libtpcf.so"

TPCF_OK = 0
TPCF_WARN_EMPTY_BIN = 1
TPCF_ERR_ARG = -1
TPCF_ERR_RANGE = -2
TPCF_ERR_CUDA = -3
TPCF_ERR_NOMEM = -4
TPCF_ERR_TIMEOUT = -5
TPCF_ERR_STATE = -6

TPCF_PERIODIC, TPCF_OPEN = 0, 1
TPCF_LOS_X, TPCF_LOS_MIDPOINT = 0, 1
TPCF_DD, TPCF_DR, TPCF_RR = 1, 2, 4
TPCF_BATCHED, TPCF_PER_LAUNCH, TPCF_HOST_INPUT = 0, 1, 2
TPCF_FP64, TPCF_TF32X3, TPCF_BF16X3 = 0, 1, 2
TPCF_OPT_GRAPHS, TPCF_OPT_AUTOTUNE, TPCF_OPT_KERNEL, TPCF_OPT_WAIT_LIMIT, TPCF_OPT_TEST_SKIP_MMA = 1, 2, 3, 4, 5
TPCF_OPT_HOST_GROUP_KB = 6
TPCF_KERNEL_AUTO, TPCF_KERNEL_DIRECT, TPCF_KERNEL_GENERAL = 0, 1, 2

EXPORTED = ("tpcf_create", "tpcf_destroy", "tpcf_sync", "tpcf_last_error", "tpcf_count", "tpcf_ls",
            "tpcf_lc_cov", "tpcf_last_count_info", "tpcf_set_timing", "tpcf_set_cell_subdiv", "tpcf_thresholds",
            "tpcf_lc_cov_noalloc", "tpcf_set_option", "tpcf_sample_cov", "tpcf_rebin_counts", "tpcf_project",
            "tpcf_multipole_matrix", "tpcf_covcov_var", "tpcf_chi2_predict", "tpcf_chi2", "tpcf_eigvalsh")


class TpcfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tpcf error {code}: {msg}")
        self.code = code


class TpcfArgError(TpcfError, ValueError):
    """An argument refused by the binding before anything reaches the library or the GPU.

    The C ABI receives raw pointers and cannot know buffer sizes, so the
    binding checks every tensor's dtype, shape, contiguity and device first."""

    def __init__(self, msg: str):
        super().__init__(TPCF_ERR_ARG, msg)


_U32 = (torch.int32, getattr(torch, "uint32", torch.int32))


def _need(t, name, dtypes, shape, device=None, optional=False):
    """Check one tensor argument: dtype in `dtypes`, exact `shape` (None entries match any size),
    contiguous, on `device` when given."""
    if t is None:
        if optional:
            return
        raise TpcfArgError(f"{name} is required")
    if not isinstance(t, torch.Tensor):
        raise TpcfArgError(f"{name} must be a torch tensor")
    if t.dtype not in dtypes:
        raise TpcfArgError(f"{name} must have dtype {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
    if t.dim() != len(shape) or any(w is not None and int(g) != int(w) for g, w in zip(t.shape, shape)):
        want = "[" + ", ".join("*" if w is None else str(w) for w in shape) + "]"
        raise TpcfArgError(f"{name} must have shape {want}, got {list(t.shape)}")
    if not t.is_contiguous():
        raise TpcfArgError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise TpcfArgError(f"{name} is on {t.device}, expected {device}")


def validate_count_args(mocks, nbin, device, out=None):
    """Checks tpcf_count's mocks (and `out`) before the call; returns (host, M).

    Each mock: exactly one of 'data' (float64 [n_d, 3]) / 'data_u32' (32-bit [3, n_d]), and for the
    randoms one of 'randoms' (float64 [n_r, 3]) / 'randoms_u32' (32-bit [3, n_r]) with 'offsets'
    (M + 1 integers, offsets[0] == 0, non-decreasing, offsets[-1] == n_r).  The catalogues are all
    on `device` or all on the host; every mock has the same M."""
    cats = [t for m in mocks for t in (m.get("data"), m.get("data_u32"), m.get("randoms"), m.get("randoms_u32"))
            if t is not None]
    for t in cats:
        if not isinstance(t, torch.Tensor):
            raise TpcfArgError("catalogues must be torch tensors")
    host = bool(cats) and not any(t.is_cuda for t in cats)
    where = torch.device("cpu") if host else device
    M = None
    for i, m in enumerate(mocks):
        d, du, r, ru = m.get("data"), m.get("data_u32"), m.get("randoms"), m.get("randoms_u32")
        if d is not None and du is not None:
            raise TpcfArgError(f"mock {i}: give one of 'data' and 'data_u32'")
        if r is not None and ru is not None:
            raise TpcfArgError(f"mock {i}: give one of 'randoms' and 'randoms_u32'")
        if d is not None:
            _need(d, f"mock {i} data", (torch.float64,), (None, 3), where)
        if du is not None:
            _need(du, f"mock {i} data_u32", _U32, (3, None), where)
        n_r = 0
        if r is not None:
            _need(r, f"mock {i} randoms", (torch.float64,), (None, 3), where)
            n_r = int(r.shape[0])
        if ru is not None:
            _need(ru, f"mock {i} randoms_u32", _U32, (3, None), where)
            n_r = int(ru.shape[1])
        offs = [int(x) for x in m.get("offsets", [0])]
        if len(offs) < 1 or offs[0] != 0:
            raise TpcfArgError(f"mock {i}: offsets must start at 0")
        if any(b < a for a, b in zip(offs, offs[1:])):
            raise TpcfArgError(f"mock {i}: offsets must be non-decreasing")
        if offs[-1] != n_r:
            raise TpcfArgError(f"mock {i}: offsets[-1] = {offs[-1]} but the randoms hold {n_r} points")
        if M is not None and len(offs) - 1 != M:
            raise TpcfArgError(f"mock {i}: every mock needs the same number of random subsets")
        M = len(offs) - 1
    M = M or 0
    if out is not None:
        n_mock = len(mocks)
        _need(out.get("dd"), "out['dd']", (torch.int64,), (n_mock, nbin), device, optional=True)
        for k in ("dr", "rr"):
            _need(out.get(k), f"out['{k}']", (torch.int64,), (n_mock, max(M, 1), nbin), device, optional=True)
    return host, M


class tpcf_binning(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("box_L", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("los", ctypes.c_int), ("observer", ctypes.c_double * 3), ("n_s", ctypes.c_int),
                ("s_edges", ctypes.POINTER(ctypes.c_double)), ("n_mu", ctypes.c_int)]


class tpcf_mock(ctypes.Structure):
    _fields_ = [("data_xyz", ctypes.c_void_p), ("data_u32", ctypes.c_void_p), ("n_d", ctypes.c_int64),
                ("rand_xyz", ctypes.c_void_p), ("rand_u32", ctypes.c_void_p),
                ("rand_offsets", ctypes.POINTER(ctypes.c_int64)), ("M", ctypes.c_int)]


class tpcf_count_info(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int64), ("n_binned", ctypes.c_int64), ("n_exact", ctypes.c_int64),
                ("n_units", ctypes.c_int64), ("paircount_ms", ctypes.c_double),
                ("n_paircount_launches", ctypes.c_int), ("cell_subdiv", ctypes.c_int),
                ("cells_per_axis", ctypes.c_int), ("n_kernels", ctypes.c_int), ("timed_calls", ctypes.c_int),
                ("unit_chunk", ctypes.c_int), ("graph_replay", ctypes.c_int), ("pair_kernel", ctypes.c_int),
                ("pair_blocks", ctypes.c_int), ("idle_frac", ctypes.c_double), ("call_ms", ctypes.c_double),
                ("stage_ms", ctypes.c_double)]


def load_library() -> ctypes.CDLL:
    """Load libtpcf.so and declare its signatures (no CUDA call is made)."""
    if not _LIBPATH.exists():
        raise ImportError(f"{_LIBPATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(str(_LIBPATH))
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.tpcf_create.argtypes = [ctypes.POINTER(P), I]
    lib.tpcf_destroy.argtypes = [P]
    lib.tpcf_destroy.restype = None
    lib.tpcf_sync.argtypes = [P, P]
    lib.tpcf_last_error.argtypes = [P]
    lib.tpcf_last_error.restype = ctypes.c_char_p
    lib.tpcf_count.argtypes = [P, ctypes.POINTER(tpcf_mock), I, ctypes.POINTER(tpcf_binning), ctypes.c_uint,
                               P, P, P, I, P]
    lib.tpcf_ls.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), I, I, I,
                            ctypes.POINTER(ctypes.c_int), I, P, P]
    lib.tpcf_lc_cov.argtypes = [P, P, P, P, I, I, I, D, I, P, P, P, P, P, P]
    lib.tpcf_last_count_info.argtypes = [P, ctypes.POINTER(tpcf_count_info)]
    lib.tpcf_set_timing.argtypes = [P, I]
    lib.tpcf_set_cell_subdiv.argtypes = [P, I]
    lib.tpcf_thresholds.argtypes = [P, ctypes.POINTER(tpcf_binning), ctypes.POINTER(ctypes.c_uint64)]
    lib.tpcf_lc_cov_noalloc.argtypes = [P, P, P, I, I, I, D, P, P, P, P, P, P]
    lib.tpcf_lc_cov_noalloc.restype = ctypes.c_int
    lib.tpcf_set_option.argtypes = [P, I, I]
    lib.tpcf_set_option.restype = ctypes.c_int
    lib.tpcf_sample_cov.argtypes = [P, P, I, I, I, P, P]
    lib.tpcf_sample_cov.restype = ctypes.c_int
    lib.tpcf_rebin_counts.argtypes = [P, P, ctypes.c_int64, I, I, I, I, P, P]
    lib.tpcf_rebin_counts.restype = ctypes.c_int
    lib.tpcf_project.argtypes = [P, P, I, I, P, I, P, P]
    lib.tpcf_project.restype = ctypes.c_int
    lib.tpcf_multipole_matrix.argtypes = [I, I, P, I, P]
    lib.tpcf_multipole_matrix.restype = ctypes.c_int
    lib.tpcf_covcov_var.argtypes = [P, P, P, I, I, D, I, P, P]
    lib.tpcf_chi2_predict.argtypes = [P, P, P, P, I, I, D, P, P]
    lib.tpcf_chi2.argtypes = [P, P, P, P, I, P, P]
    lib.tpcf_eigvalsh.argtypes = [P, P, I, P, P]
    for name in ("tpcf_covcov_var", "tpcf_chi2_predict", "tpcf_chi2", "tpcf_eigvalsh"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("tpcf_create", "tpcf_sync", "tpcf_count", "tpcf_ls", "tpcf_lc_cov", "tpcf_last_count_info",
                 "tpcf_set_timing", "tpcf_set_cell_subdiv", "tpcf_thresholds"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_binning(s_edges, n_mu=1, geometry=TPCF_PERIODIC, box_L=1.0, origin=(0.0, 0.0, 0.0), los=TPCF_LOS_X,
                 observer=(0.0, 0.0, 0.0)):
    """tpcf_binning; the returned object keeps the edge array alive."""
    edges = (ctypes.c_double * len(s_edges))(*[float(e) for e in s_edges])
    b = tpcf_binning(int(geometry), float(box_L), (ctypes.c_double * 3)(*origin), int(los),
                     (ctypes.c_double * 3)(*observer), len(s_edges) - 1,
                     ctypes.cast(edges, ctypes.POINTER(ctypes.c_double)), int(n_mu))
    b._edges = edges
    return b


def tpcf_thresholds(binning) -> list:
    """Exact integer s-bin thresholds used by tpcf_count (host computation, no GPU)."""
    T = (ctypes.c_uint64 * (binning.n_s + 1))()
    rc = lib().tpcf_thresholds(None, ctypes.byref(binning), T)
    if rc != TPCF_OK:
        raise TpcfError(rc, "tpcf_thresholds failed")
    return [int(t) for t in T]


def tpcf_multipole_matrix(n_s, n_mu, ells=(0, 2, 4)):
    """Legendre multipole matrix [len(ells) * n_s, n_s * n_mu] (float64 numpy, host computation)."""
    import numpy as np
    ls = (ctypes.c_int * len(ells))(*[int(x) for x in ells])
    P = np.empty((len(ells) * n_s, n_s * n_mu), dtype=np.float64)
    rc = lib().tpcf_multipole_matrix(int(n_s), int(n_mu), ls, len(ells), ctypes.c_void_p(P.ctypes.data))
    if rc != TPCF_OK:
        raise TpcfError(rc, "tpcf_multipole_matrix failed")
    return P


class Context:
    """A libtpcf context on one CUDA device (tpcf_create / tpcf_destroy)."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        self.device = int(device)
        h = ctypes.c_void_p()
        rc = self._lib.tpcf_create(ctypes.byref(h), self.device)
        if rc != TPCF_OK:
            raise TpcfError(rc, "tpcf_create failed")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._lib.tpcf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc < 0:
            raise TpcfError(rc, self._lib.tpcf_last_error(self.handle).decode())
        return rc

    # -- C entry points, same names -------------------------------------------------

    def tpcf_sync(self, stream=None) -> int:
        return self._check(self._lib.tpcf_sync(self.handle, _stream(stream)))

    def tpcf_set_timing(self, enable: bool):
        self._check(self._lib.tpcf_set_timing(self.handle, int(bool(enable))))

    def tpcf_set_cell_subdiv(self, subdiv: int):
        self._check(self._lib.tpcf_set_cell_subdiv(self.handle, int(subdiv)))

    def tpcf_set_option(self, option: int, value: int):
        self._check(self._lib.tpcf_set_option(self.handle, int(option), int(value)))

    def tpcf_last_count_info(self) -> dict:
        info = tpcf_count_info()
        self._check(self._lib.tpcf_last_count_info(self.handle, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def tpcf_count(self, mocks, binning, terms=TPCF_DD | TPCF_DR | TPCF_RR, mode=TPCF_BATCHED, stream=None,
                   out=None):
        """Pair counts of every mock.

        mocks: sequence of dicts with keys
          'data' (float64 [n_d,3]) or 'data_u32' (int32/uint32 [3,n_d]),
          'randoms' (float64 [n_r,3]) or 'randoms_u32' ([3,n_r]), 'offsets' (M+1 ints).
        The catalogues are either all CUDA tensors or all CPU tensors (pinned
        for an asynchronous copy): CPU tensors are passed as host arrays with
        TPCF_HOST_INPUT, and the library copies them in on the stream.
        Returns dict of int64 CUDA tensors dd [n_mock,nbin], dr/rr [n_mock,M,nbin].
        """
        n_mock = len(mocks)
        nbin = binning.n_s * binning.n_mu
        arr = (tpcf_mock * max(1, n_mock))()
        keep = []
        dev = torch.device("cuda", self.device)
        host, M = validate_count_args(mocks, nbin, dev, out)
        if host:
            mode = int(mode) | TPCF_HOST_INPUT
        for i, m in enumerate(mocks):
            d = m.get("data")
            du = m.get("data_u32")
            r = m.get("randoms")
            ru = m.get("randoms_u32")
            offs = m.get("offsets", [0])
            o = (ctypes.c_int64 * len(offs))(*[int(x) for x in offs])
            keep.append(o)
            n_d = d.shape[0] if d is not None else (du.shape[1] if du is not None else 0)
            arr[i] = tpcf_mock(_ptr(d), _ptr(du), n_d, _ptr(r), _ptr(ru),
                               ctypes.cast(o, ctypes.POINTER(ctypes.c_int64)), M)
        if out is None:
            out = {"dd": torch.empty((n_mock, nbin), dtype=torch.int64, device=dev),
                   "dr": torch.empty((n_mock, max(M, 1), nbin), dtype=torch.int64, device=dev),
                   "rr": torch.empty((n_mock, max(M, 1), nbin), dtype=torch.int64, device=dev)}
        rc = self._lib.tpcf_count(self.handle, arr, n_mock, ctypes.byref(binning), int(terms),
                                  _ptr(out["dd"]), _ptr(out["dr"]), _ptr(out["rr"]), int(mode), _stream(stream))
        self._check(rc)
        del keep
        return out

    def tpcf_ls(self, dd, dr, rr, n_d, n_r, sel, stream=None, out=None):
        """Split Landy-Szalay xi [n_mock, nbin] (float64 CUDA) over random subsets `sel`."""
        dev = torch.device("cuda", self.device)
        _need(dd, "dd", (torch.int64,), (None, None), dev)
        n_mock, nbin = dd.shape
        _need(dr, "dr", (torch.int64,), (n_mock, None, nbin), dev)
        M = dr.shape[1]
        _need(rr, "rr", (torch.int64,), (n_mock, M, nbin), dev)
        _need(out, "out", (torch.float64,), (n_mock, nbin), dev, optional=True)
        if len(n_d) != n_mock or len(n_r) != n_mock or any(len(row) != M for row in n_r):
            raise TpcfArgError("n_d must have n_mock entries and n_r n_mock rows of M entries")
        if not sel or any(not 0 <= int(x) < M for x in sel):
            raise TpcfArgError("sel must name subsets in [0, M)")
        nd = (ctypes.c_int64 * max(1, n_mock))(*[int(x) for x in n_d])
        flat = [int(x) for row in n_r for x in row]
        nr = (ctypes.c_int64 * max(1, len(flat)))(*flat)
        s = (ctypes.c_int * len(sel))(*[int(x) for x in sel])
        if out is None:
            out = torch.empty((n_mock, nbin), dtype=torch.float64, device=dd.device)
        rc = self._lib.tpcf_ls(self.handle, _ptr(dd), _ptr(dr), _ptr(rr), nd, nr, n_mock, M, nbin, s, len(sel),
                               _ptr(out), _stream(stream))
        self._check(rc)
        return out

    def tpcf_lc_cov(self, xi_a1, xi_a2, xi_b, M_a=1, M=math.inf, precision=TPCF_FP64, stream=None,
                    want_parts=True):
        """LC covariance (Eqs. R1R2, LCdef); returns dict of float64 CUDA [nbin, nbin] tensors."""
        dev = torch.device("cuda", self.device)
        _need(xi_a1, "xi_a1", (torch.float64,), (None, None), dev)
        n_mock, nbin = xi_a1.shape
        _need(xi_a2, "xi_a2", (torch.float64,), (n_mock, nbin), dev)
        _need(xi_b, "xi_b", (torch.float64,), (n_mock, nbin), dev)
        mk = lambda: torch.empty((nbin, nbin), dtype=torch.float64, device=dev)
        out = {"C_lc": mk()}
        if want_parts:
            out.update(Ca=mk(), Cb=mk(), A=mk(), B=mk())
        rc = self._lib.tpcf_lc_cov(self.handle, _ptr(xi_a1), _ptr(xi_a2), _ptr(xi_b), n_mock, nbin, int(M_a),
                                   float(M), int(precision), _ptr(out["C_lc"]), _ptr(out.get("Ca")),
                                   _ptr(out.get("Cb")), _ptr(out.get("A")), _ptr(out.get("B")), _stream(stream))
        self._check(rc)
        return out

    def tpcf_rebin_counts(self, counts, n_s, n_mu, f_s, f_mu, stream=None):
        """Counts [..., n_s * n_mu] (int64 CUDA) summed into [..., (n_s/f_s) * (n_mu/f_mu)] wider bins."""
        if not isinstance(counts, torch.Tensor) or counts.dim() < 1:
            raise TpcfArgError("counts must be an int64 tensor [..., n_s * n_mu]")
        _need(counts, "counts", (torch.int64,), (None,) * counts.dim(), torch.device("cuda", self.device))
        if counts.shape[-1] != int(n_s) * int(n_mu):
            raise TpcfArgError(f"counts must end in n_s * n_mu = {int(n_s) * int(n_mu)} bins")
        lead = tuple(counts.shape[:-1])
        rows = 1
        for d in lead:
            rows *= int(d)
        out = torch.empty(lead + ((n_s // max(1, f_s)) * (n_mu // max(1, f_mu)),), dtype=torch.int64,
                          device=counts.device)
        self._check(self._lib.tpcf_rebin_counts(self.handle, _ptr(counts), rows, int(n_s), int(n_mu), int(f_s),
                                                int(f_mu), _ptr(out), _stream(stream)))
        return out

    def tpcf_project(self, P, xi, stream=None):
        """xi [n_mock, nbin] mapped by P [n_out, nbin] (float64 CUDA): returns [n_mock, n_out]."""
        dev = torch.device("cuda", self.device)
        _need(P, "P", (torch.float64,), (None, None), dev)
        n_out, nbin = P.shape
        _need(xi, "xi", (torch.float64,), (None, nbin), dev)
        n_mock = xi.shape[0]
        y = torch.empty((n_mock, n_out), dtype=torch.float64, device=xi.device)
        self._check(self._lib.tpcf_project(self.handle, _ptr(P), n_out, nbin, _ptr(xi), n_mock, _ptr(y),
                                           _stream(stream)))
        return y

    def tpcf_covcov_var(self, A, B, n_mock, M_a=1, M=math.inf, stream=None):
        """Var(C_ij) [nbin, nbin]: LC form from (A, B), or the sample-covariance form from C = A when B is None."""
        dev = torch.device("cuda", self.device)
        _need(A, "A", (torch.float64,), (None, None), dev)
        nbin = A.shape[0]
        _need(A, "A", (torch.float64,), (nbin, nbin), dev)
        _need(B, "B", (torch.float64,), (nbin, nbin), dev, optional=True)
        var = torch.empty((nbin, nbin), dtype=torch.float64, device=A.device)
        self._check(self._lib.tpcf_covcov_var(self.handle, _ptr(A), _ptr(B), nbin, int(M_a), float(M), int(n_mock),
                                              _ptr(var), _stream(stream)))
        return var

    def tpcf_chi2_predict(self, A, B, C_ref, M_a=1, M=math.inf, stream=None):
        """Predicted <chi^2_2> (device scalar tensor) of the LC (B given) or sample (B None) covariance."""
        dev = torch.device("cuda", self.device)
        _need(A, "A", (torch.float64,), (None, None), dev)
        nbin = A.shape[0]
        _need(A, "A", (torch.float64,), (nbin, nbin), dev)
        _need(B, "B", (torch.float64,), (nbin, nbin), dev, optional=True)
        _need(C_ref, "C_ref", (torch.float64,), (nbin, nbin), dev)
        out = torch.empty((), dtype=torch.float64, device=A.device)
        self._check(self._lib.tpcf_chi2_predict(self.handle, _ptr(A), _ptr(B), _ptr(C_ref), A.shape[0], int(M_a),
                                                float(M), _ptr(out), _stream(stream)))
        return out

    def tpcf_chi2(self, C_est, C_true, C_ref, stream=None):
        """chi^2 of Eq. (chi2) (device scalar tensor)."""
        dev = torch.device("cuda", self.device)
        _need(C_est, "C_est", (torch.float64,), (None, None), dev)
        nbin = C_est.shape[0]
        for t, nm in ((C_est, "C_est"), (C_true, "C_true"), (C_ref, "C_ref")):
            _need(t, nm, (torch.float64,), (nbin, nbin), dev)
        out = torch.empty((), dtype=torch.float64, device=C_est.device)
        self._check(self._lib.tpcf_chi2(self.handle, _ptr(C_est), _ptr(C_true), _ptr(C_ref), C_est.shape[0],
                                        _ptr(out), _stream(stream)))
        return out

    def tpcf_eigvalsh(self, C, stream=None):
        """Ascending eigenvalues of the symmetric float64 CUDA matrix C."""
        dev = torch.device("cuda", self.device)
        _need(C, "C", (torch.float64,), (None, None), dev)
        n = C.shape[0]
        _need(C, "C", (torch.float64,), (n, n), dev)
        w = torch.empty((n,), dtype=torch.float64, device=C.device)
        self._check(self._lib.tpcf_eigvalsh(self.handle, _ptr(C), n, _ptr(w), _stream(stream)))
        return w

    def tpcf_sample_cov(self, xi, precision=TPCF_FP64, stream=None):
        """Sample covariance of xi [n_mock, nbin] over the mocks (Eq. bruteforce); float64 CUDA [nbin, nbin]."""
        _need(xi, "xi", (torch.float64,), (None, None), torch.device("cuda", self.device))
        n_mock, nbin = xi.shape
        C = torch.empty((nbin, nbin), dtype=torch.float64, device=xi.device)
        self._check(self._lib.tpcf_sample_cov(self.handle, _ptr(xi), n_mock, nbin, int(precision), _ptr(C),
                                              _stream(stream)))
        return C
