"""CPU oracle for the linear-construction (LC) covariance hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never calls it, and it never
calls the product path.

It is the plain definition of what the method computes, written for
checkability rather than speed:

* ``quantize``   -- positions to integer grid coordinates (the exact-count
                    convention shared with the GPU path; the paper is silent
                    on coordinate precision).
* ``thresholds`` -- squared s-bin edges in grid units, rounded up to
                    integers, in exact rational arithmetic.
* ``count_pairs`` / ``count_mock`` -- brute-force O(N^2) DD, DR_i and RR_i
                    counts of Sect. 2.1 with the (r, mu) binning of Sect. 4.3
                    (C with OpenMP, ``bruteforce.c``).
* ``ls``         -- the split Landy-Szalay estimator of Sect. 2.1 in float64.
* ``sample_cov`` -- the sample covariance, Eq. (bruteforce), two-pass float64.
* ``lc_cov``     -- the linear construction: Eqs. (R1R2) and (LCdef).
* ``cov_ab``     -- the two-size decomposition of Eq. (CovAB).
* ``covcov_var`` / ``chi2_predict`` / ``chi2`` / ``eigvalsh`` -- accuracy of
                    the covariance estimates (Sect. 3, Sect. 5.3).
* ``rebin_counts`` / ``multipole_matrix`` / ``project`` -- the linear maps
                    applied before the covariance (Sect. 2.3, Sect. 4.3):
                    bins combined into wider ones, the Legendre multipoles.

Readings of the paper where it is silent (all listed in the design notes):
bins are half-open [e_k, e_{k+1}); mu is |cos| in [0, 1] with the top bin
closed; the random normalisations use the actual subset sizes N_r,i, which
equals the paper's N_d form when N_r,i = N_d; rr = 0 gives xi = NaN.  In
Eq. (covcov_fast) D = A + B / (2 M_a) (derived from Eqs. covcov and Cfastx;
the printed D = A + B / M_a contradicts Eq. covcov_fast2).
"""
from __future__ import annotations

import ctypes
import math
import os
import pathlib
import subprocess
from fractions import Fraction

import numpy as np

PERIODIC, OPEN = 0, 1
LOS_X, LOS_MIDPOINT = 0, 1

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "bruteforce.c"
_BUILD = _HERE / "_build"
_LIB = None
_EMPTY = np.zeros((3, 1), dtype=np.uint32)  # stands in for an empty catalogue


def build(force: bool = False) -> pathlib.Path:
    """Compile the brute-force counter with gcc (plain C + OpenMP)."""
    _BUILD.mkdir(exist_ok=True)
    so = _BUILD / "libtpcf_oracle.so"
    if force or not so.exists() or so.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = so.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall",
                        "-o", str(tmp), str(_SRC)], check=True)
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(str(build()))
        f = lib.oracle_count_pairs
        P = ctypes.c_void_p
        f.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P,
                      ctypes.c_int, P, ctypes.c_int, P, P]
        f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


# ---------------------------------------------------------------------------
# Geometry and binning
# ---------------------------------------------------------------------------

def grid_scale(geometry: int, L: float) -> Fraction:
    """Grid units per unit length: 2^32/L (periodic box side L) or 2^30/L (open bounding cube side L)."""
    bits = 32 if geometry == PERIODIC else 30
    return Fraction(2 ** bits) / Fraction(float(L))


def quantize(xyz, geometry: int, L: float, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Positions float64 [n][3] -> grid coordinates uint32 [3][n].

    periodic: t = x / L; t -= floor(t); u = floor(t * 2^32), and 2^32 wraps to 0.
    open:     t = (x - x0) / L must lie in [0, 1); u = floor(t * 2^30).
    Each step is one IEEE double operation, so the result is reproducible.
    """
    x = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.empty((3, x.shape[0]), dtype=np.uint32)
    for c in range(3):
        if geometry == PERIODIC:
            t = x[:, c] / np.float64(L)
            t = t - np.floor(t)
            v = np.floor(t * np.float64(2.0 ** 32))
            v[v >= 2.0 ** 32] -= 2.0 ** 32
        else:
            t = (x[:, c] - np.float64(origin[c])) / np.float64(L)
            if np.any(~(t >= 0.0)) or np.any(~(t < 1.0)):
                raise ValueError("open geometry: a position lies outside the bounding cube")
            v = np.floor(t * np.float64(2.0 ** 30))
        out[c] = v.astype(np.uint64).astype(np.uint32)
    return out


def quantize_observer(observer, L: float, origin=(0.0, 0.0, 0.0)) -> list:
    """Observer position in open-geometry grid units (floor, may lie outside the cube)."""
    return [int(math.floor(((float(observer[c]) - float(origin[c])) / float(L)) * 2.0 ** 30))
            for c in range(3)]


def thresholds(s_edges, geometry: int, L: float) -> list:
    """T_k = ceil(e_k^2 q^2) as exact integers, q the grid scale.

    A pair with squared grid separation D2 lies in s-bin k iff T_k <= D2 < T_{k+1},
    i.e. e_k <= sqrt(D2)/q < e_{k+1}.
    """
    q = grid_scale(geometry, L)
    out = []
    for e in s_edges:
        v = Fraction(float(e)) ** 2 * q * q
        out.append(-((-v.numerator) // v.denominator))  # ceil
    return out


class Binning:
    """Validated binning and geometry (plain Python ints for exact bounds)."""

    def __init__(self, s_edges, n_mu: int = 1, geometry: int = PERIODIC, L: float = 1.0,
                 origin=(0.0, 0.0, 0.0), los: int = LOS_X, observer=(0.0, 0.0, 0.0)):
        self.s_edges = [float(e) for e in s_edges]
        self.n_s = len(self.s_edges) - 1
        self.n_mu = int(n_mu)
        self.geometry = int(geometry)
        self.L = float(L)
        self.origin = tuple(float(o) for o in origin)
        self.los = int(los)
        self.observer = tuple(float(o) for o in observer)
        if self.n_s < 1 or self.n_mu < 1:
            raise ValueError("need at least one s bin and one mu bin")
        if any(not (b > a) for a, b in zip(self.s_edges, self.s_edges[1:])) or self.s_edges[0] < 0:
            raise ValueError("s edges must be non-negative and strictly increasing")
        if not (self.L > 0):
            raise ValueError("box side must be positive")
        if self.geometry == PERIODIC:
            if not (self.s_edges[-1] < self.L / 2):
                raise ValueError("periodic box: s_max must be below L/2 (unique minimum image)")
            if self.n_mu > 1 and self.los != LOS_X:
                raise ValueError("periodic box supports the plane-parallel (x) line of sight only")
        self.T = thresholds(self.s_edges, self.geometry, self.L)
        self.obs_u = [0, 0, 0]
        if self.geometry == OPEN and self.los == LOS_MIDPOINT:
            self.obs_u = quantize_observer(self.observer, self.L, self.origin)
        self._check_width()

    @property
    def nbin(self) -> int:
        return self.n_s * self.n_mu

    def _check_width(self):
        d2max = self.T[-1] - 1
        if d2max >= 2 ** 63:
            raise ValueError("separation range too large for 64-bit squared distances")
        if self.n_mu > 1:
            if self.los == LOS_X:
                lmax2 = 1
            else:
                top = 2 ** 31 - 2
                lmax2 = sum(max(abs(2 * o), abs(top - 2 * o)) ** 2 for o in self.obs_u)
            if self.n_mu * self.n_mu * d2max * lmax2 >= 2 ** 127:
                raise ValueError("mu test exceeds 128-bit range for this geometry")


# ---------------------------------------------------------------------------
# Pair counts (Sect. 2.1, Sect. 4.3)
# ---------------------------------------------------------------------------

def count_pairs(ua: np.ndarray, ub, binning: Binning):
    """Brute-force histogram of pairs between grid catalogues ua [3][na] and ub [3][nb].

    ub is None: unordered pairs within ua (auto count, DD or RR_i).
    Returns (hist int64 [n_s * n_mu], unbinned pair count).
    """
    ua = np.ascontiguousarray(ua, dtype=np.uint32)
    na = ua.shape[1]
    if ub is not None:
        ub = np.ascontiguousarray(ub, dtype=np.uint32)
        nb = ub.shape[1]
    else:
        nb = 0
    hist = np.zeros(binning.nbin, dtype=np.int64)
    unb = np.zeros(1, dtype=np.int64)
    T = np.array(binning.T, dtype=np.uint64)
    obs = np.array(binning.obs_u, dtype=np.int64)
    rc = _lib().oracle_count_pairs(
        (ua if na else _EMPTY).ctypes.data, na,
        (ub if nb else _EMPTY).ctypes.data if ub is not None else None, nb,
        binning.geometry, binning.los, obs.ctypes.data,
        binning.n_s, T.ctypes.data, binning.n_mu, hist.ctypes.data, unb.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return hist, int(unb[0])


def count_mock(data_xyz, rand_xyz_subsets, binning: Binning, terms=("DD", "DR", "RR")):
    """DD, DR_i and RR_i counts for one mock (Sect. 2.1).

    Returns dict with 'DD' [nbin], 'DR' [M][nbin], 'RR' [M][nbin] (int64).
    """
    qd = quantize(data_xyz, binning.geometry, binning.L, binning.origin)
    qr = [quantize(r, binning.geometry, binning.L, binning.origin) for r in rand_xyz_subsets]
    return count_mock_u32(qd, qr, binning, terms)


def count_mock_u32(qd, qr, binning: Binning, terms=("DD", "DR", "RR")):
    M = len(qr)
    out = {"DD": np.zeros(binning.nbin, np.int64),
           "DR": np.zeros((M, binning.nbin), np.int64),
           "RR": np.zeros((M, binning.nbin), np.int64)}
    if "DD" in terms:
        out["DD"] = count_pairs(qd, None, binning)[0]
    for i, r in enumerate(qr):
        if "DR" in terms:
            out["DR"][i] = count_pairs(qd, r, binning)[0]
        if "RR" in terms:
            out["RR"][i] = count_pairs(r, None, binning)[0]
    return out


# ---------------------------------------------------------------------------
# Split Landy-Szalay estimator (Sect. 2.1)
# ---------------------------------------------------------------------------

def ls(DD, DR, RR, n_d: int, n_r, sel) -> np.ndarray:
    """Split Landy-Szalay estimate over the random subsets listed in ``sel``.

    dd = DD / (N_d (N_d - 1) / 2)
    dr = (1/|S|) sum_{i in S} DR_i / (N_d N_r,i)
    rr = (1/|S|) sum_{i in S} RR_i / (N_r,i (N_r,i - 1) / 2)
    xi = (dd - 2 dr) / rr + 1          (NaN where rr == 0)
    Works on one mock (DD [nbin], DR/RR [M][nbin]) in float64.
    """
    DD = np.asarray(DD, dtype=np.float64)
    DR = np.asarray(DR, dtype=np.float64)
    RR = np.asarray(RR, dtype=np.float64)
    n_d = float(n_d)
    dd = DD / (n_d * (n_d - 1.0) / 2.0)
    dr = np.zeros_like(dd)
    rr = np.zeros_like(dd)
    for i in sel:
        nr = float(n_r[i])
        dr += DR[i] / (n_d * nr)
        rr += RR[i] / (nr * (nr - 1.0) / 2.0)
    dr /= len(sel)
    rr /= len(sel)
    with np.errstate(divide="ignore", invalid="ignore"):
        xi = (dd - 2.0 * dr) / rr + 1.0
    xi[rr == 0] = np.nan
    return xi


# ---------------------------------------------------------------------------
# Covariances (Sect. 2.2-2.3)
# ---------------------------------------------------------------------------

def sample_cov(xi) -> np.ndarray:
    """Sample covariance, Eq. (bruteforce): 1/(N-1) sum_i (xi_i - mean)(xi_i - mean)^T.

    xi is [N mocks][nbin]; two passes (mean first, then centred products).
    """
    x = np.asarray(xi, dtype=np.float64)
    n = x.shape[0]
    if n < 2:
        raise ValueError("sample covariance needs at least two mocks")
    mean = x.sum(axis=0) / n
    r = x - mean
    return (r.T @ r) / (n - 1)


def lc_cov(xi_a1, xi_a2, xi_b, M_a: int, M: float) -> dict:
    """Linear construction covariance, Eqs. (R1R2) and (LCdef).

    C^a = (C[xi(D,R1)] + C[xi(D,R2)]) / 2        (random catalogue size M_a)
    C^b = C[xi(D, R1 u R2)]                       (size 2 M_a, split estimator)
    A   = 2 C^b - C^a
    B   = 2 M_a (C^a - C^b)
    C^LC = A + B / M        (M = inf gives A)
    """
    Ca = 0.5 * sample_cov(xi_a1) + 0.5 * sample_cov(xi_a2)
    Cb = sample_cov(xi_b)
    A = 2.0 * Cb - Ca
    B = 2.0 * M_a * (Ca - Cb)
    C = A + B / float(M)
    return {"Ca": Ca, "Cb": Cb, "A": A, "B": B, "C_lc": C}


def cov_ab(C_Ma, C_Mb, M_a: float, M_b: float):
    """Eq. (CovAB): A and B from covariances measured at two random-catalogue sizes M_a < M_b."""
    C_Ma = np.asarray(C_Ma, dtype=np.float64)
    C_Mb = np.asarray(C_Mb, dtype=np.float64)
    A = (M_b / (M_b - M_a)) * C_Mb - (M_a / (M_b - M_a)) * C_Ma
    B = (M_a * M_b / (M_b - M_a)) * (C_Ma - C_Mb)
    return A, B


# ---------------------------------------------------------------------------
# Linear maps of the correlation function (Sect. 2.3, Sect. 4.3)
# ---------------------------------------------------------------------------

def rebin_counts(counts, n_s: int, n_mu: int, f_s: int, f_mu: int) -> np.ndarray:
    """Pair counts [..., n_s * n_mu] combined into wider bins: groups of f_s
    consecutive s bins and f_mu consecutive mu bins are summed."""
    c = np.asarray(counts, dtype=np.int64)
    if n_s % f_s or n_mu % f_mu:
        raise ValueError("re-binning factors must divide the bin counts")
    lead = c.shape[:-1]
    out = np.zeros(lead + (n_s // f_s, n_mu // f_mu), dtype=np.int64)
    c = c.reshape(lead + (n_s, n_mu))
    for k in range(n_s):
        for j in range(n_mu):
            out[..., k // f_s, j // f_mu] += c[..., k, j]
    return out.reshape(lead + ((n_s // f_s) * (n_mu // f_mu),))


def multipole_matrix(n_s: int, n_mu: int, ells=(0, 2, 4)) -> np.ndarray:
    """Matrix of the Legendre multipoles xi_l(s) = (2l+1)/2 int_{-1}^{1} xi(s, mu) P_l(mu) dmu
    (Sect. 4.3) for xi binned in n_s x n_mu uniform |mu| bins on [0, 1].

    xi(s, mu) is constant on each bin and depends on |mu|, so bin j of |mu|
    covers [mu_j, mu_{j+1}] and [-mu_{j+1}, -mu_j]; the integral of P_l over
    both pieces comes from numpy's Legendre antiderivative.
    Rows (ell index, s bin), columns (s bin, mu bin).
    """
    from numpy.polynomial import legendre as npl
    edges = np.arange(n_mu + 1, dtype=np.float64) / n_mu
    P = np.zeros((len(ells) * n_s, n_s * n_mu))
    for i, ell in enumerate(ells):
        anti = npl.Legendre.basis(ell).integ()
        for j in range(n_mu):
            a, b = edges[j], edges[j + 1]
            integral = (anti(b) - anti(a)) + (anti(-a) - anti(-b))
            for k in range(n_s):
                P[i * n_s + k, k * n_mu + j] = (2 * ell + 1) / 2.0 * integral
    return P


def project(P, xi) -> np.ndarray:
    """Every mock's xi row mapped by P: y[m] = P xi[m]."""
    return np.asarray(xi, dtype=np.float64) @ np.asarray(P, dtype=np.float64).T


# ---------------------------------------------------------------------------
# Accuracy of the covariance estimates (Sect. 3, Sect. 5.3)
# ---------------------------------------------------------------------------

def covcov_var(A, B, n_mock: int, M_a: int = 1, M: float = math.inf) -> np.ndarray:
    """Variance of every covariance element for Gaussian xi (k = i, l = j of the
    covariance of covariance).

    B given: the LC covariance, Eq. (covcov_fast),
      (N-1) Var(C_ij) = D_ii D_jj + D_ij^2 + (1/(2 M_a) - 1/M)^2 (B_ii B_jj + B_ij^2).
    D is the covariance of (x + x')/2, the xi of the 2 M_a random catalogue:
    applying Eq. (covcov) to the four terms of Eq. (Cfastx) gives
    D = A + B / (2 M_a) (the printed A + B / M_a disagrees with Eq.
    covcov_fast2 and with the M = 2 M_a limit).
    B None: the sample covariance C = A, Eq. (covcov_brute),
      (N-1) Var(C_ij) = C_ii C_jj + C_ij^2.
    """
    A = np.asarray(A, dtype=np.float64)
    if B is None:
        D = A
        extra = np.zeros_like(A)
    else:
        B = np.asarray(B, dtype=np.float64)
        D = A + B / (2.0 * M_a)
        c = 1.0 / (2.0 * M_a) - 1.0 / float(M)
        extra = c * c * (np.outer(np.diag(B), np.diag(B)) + B * B)
    return (np.outer(np.diag(D), np.diag(D)) + D * D + extra) / (n_mock - 1)


def chi2_predict(A, B, C_ref, M_a: int = 1, M: float = math.inf) -> float:
    """Predicted <chi^2_2> (Sect. 5.3): (1/N_bin^2) sum_ij (N-1) Var(C_ij) / (R_ii R_jj)."""
    R = np.asarray(C_ref, dtype=np.float64)
    r = np.diag(R)
    v = covcov_var(A, B, 2, M_a, M)       # N = 2: (N - 1) Var
    return float(np.sum(v / np.outer(r, r)) / R.shape[0] ** 2)


def chi2(C_est, C_true, C_ref) -> float:
    """Eq. (chi2): (1/N_bin^2) sum_ij (C_est - C_true)_ij^2 / (C_ref,ii C_ref,jj)."""
    E = np.asarray(C_est, dtype=np.float64)
    T = np.asarray(C_true, dtype=np.float64)
    r = np.diag(np.asarray(C_ref, dtype=np.float64))
    return float(np.sum((E - T) ** 2 / np.outer(r, r)) / E.shape[0] ** 2)


def eigvalsh(C) -> np.ndarray:
    """Ascending eigenvalues of a symmetric matrix (LAPACK through numpy), the
    eigenspectrum check recommended before inverting an LC covariance (Sect. 3.4)."""
    return np.linalg.eigvalsh(np.asarray(C, dtype=np.float64))
