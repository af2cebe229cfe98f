"""CPU oracle for the JK build: plain FP64, McMurchie-Davidson integrals.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package. The product path
(the CUDA library and its Python binding) never imports it, and it imports
nothing from the product package.

The numerical core lives in ``jk_oracle.c`` (compiled with gcc on first use);
this module marshals numpy arrays to it and adds the Cartesian-to-spherical
transform in plain numpy.

Parity status of each function is stated in its docstring. Every function
here is pinned by ``tests/test_oracle_pins.py`` against closed forms,
independent quadrature or brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from math import factorial, sqrt, pi

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libjk_oracle.so")
_lib = None
_lock = threading.Lock()

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # JK_ORACLE_LIB points the wrapper at another build of jk_oracle.c;
        # the mutation test uses it to check that planted mistakes fail the pins.
        override = os.environ.get("JK_ORACLE_LIB")
        lib = ctypes.CDLL(override if override else build())
        lib.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        lib.oracle_boys.restype = None
        lib.oracle_eri_prim.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 4 + [_dp] * 5
        lib.oracle_eri_prim.restype = None
        lib.oracle_eri_shell.argtypes = [_ip, _dp, _dp, _dp] + [ctypes.c_int] * 4 + [_dp]
        lib.oracle_eri_shell.restype = None
        lib.oracle_schwarz.argtypes = [_ip, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.oracle_schwarz.restype = None
        lib.oracle_dmax.argtypes = [_ip, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp]
        lib.oracle_dmax.restype = None
        lib.oracle_eri_full.argtypes = [_ip, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.oracle_eri_full.restype = None
        jk_args = [_ip, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.oracle_jk_brute.argtypes = jk_args
        lib.oracle_jk_brute.restype = ctypes.c_longlong
        lib.oracle_jk_screened.argtypes = jk_args
        lib.oracle_jk_screened.restype = ctypes.c_longlong
        lib.oracle_jk_rows.argtypes = [_ip, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int,
                                       _ip, ctypes.c_int, _dp, _ip, ctypes.c_int, _dp]
        lib.oracle_jk_rows.restype = ctypes.c_longlong
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_omega.argtypes = [ctypes.c_double]
        lib.oracle_set_omega.restype = None
        _lib = lib
        return lib


class omega_operator:
    """Context: integrals of erf(w r)/r (w > 0), erfc(|w| r)/r (w < 0) or 1/r (w = 0).

    The Schwarz factors stay those of 1/r (a valid bound for both attenuated
    operators, whose Fourier transforms lie between 0 and that of 1/r)."""

    def __init__(self, omega: float):
        self.omega = float(omega)

    def __enter__(self):
        _load().oracle_set_omega(self.omega)
        _current_omega[0] = self.omega
        return self

    def __exit__(self, *exc):
        _load().oracle_set_omega(0.0)
        _current_omega[0] = 0.0
        return False


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().oracle_num_threads())


def ncart(l):
    return (l + 1) * (l + 2) // 2


def cart_components(l):
    """(lx, ly, lz) of each Cartesian component, x descending then y (Sec. 2)."""
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


# ------------------------------------------------------------------ Boys
def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt for m = 0..mmax.

    Pinned: F_m(0) = 1/(2m+1); F_0 = sqrt(pi) erf(sqrt T)/(2 sqrt T);
    independent adaptive quadrature; large-T asymptote.
    """
    out = np.zeros(mmax + 1)
    _load().oracle_boys(int(mmax), float(T), out)
    return out


# ------------------------------------------------------------ integrals
def eri_prim(ls, alphas, centers) -> np.ndarray:
    """Primitive Cartesian ERI block (a b|c d), unnormalised, coefficient 1.

    ``ls`` = (la, lb, lc, ld), ``alphas`` the four exponents, ``centers`` a
    (4, 3) array in bohr. Returns shape (ncart(la), ..., ncart(ld)).
    Pinned against the (ss|ss) closed form, the centre-derivative identity
    and an independent Gaussian-transform quadrature.
    """
    la, lb, lc, ld = (int(x) for x in ls)
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(4, 3)
    out = np.zeros(ncart(la) * ncart(lb) * ncart(lc) * ncart(ld))
    _load().oracle_eri_prim(la, lb, lc, ld, *(float(a) for a in alphas),
                            np.ascontiguousarray(c[0]), np.ascontiguousarray(c[1]),
                            np.ascontiguousarray(c[2]), np.ascontiguousarray(c[3]), out)
    return out.reshape(ncart(la), ncart(lb), ncart(lc), ncart(ld))


def _basis_args(mol):
    sh = np.ascontiguousarray(mol.shells, dtype=np.int32)
    return (sh, int(sh.shape[0]), np.ascontiguousarray(mol.coords, dtype=np.float64).ravel(),
            np.ascontiguousarray(mol.exps, dtype=np.float64),
            np.ascontiguousarray(mol.coeffs, dtype=np.float64))


def eri_shell(mol, a, b, c, d) -> np.ndarray:
    """Contracted Cartesian block (ab|cd) of eq:rys0 for shells a, b, c, d."""
    sh, nsh, xyz, ex, co = _basis_args(mol)
    ls = [int(sh[s, 1]) for s in (a, b, c, d)]
    out = np.zeros(int(np.prod([ncart(l) for l in ls])))
    _load().oracle_eri_shell(sh, xyz, ex, co, int(a), int(b), int(c), int(d), out)
    return out.reshape([ncart(l) for l in ls])


def eri_full(mol) -> np.ndarray:
    """Full Cartesian (ij|kl) tensor, every shell quartet, no screening."""
    sh, nsh, xyz, ex, co = _basis_args(mol)
    nao = int(sum(ncart(int(l)) for l in sh[:, 1]))
    out = np.zeros(nao ** 4)
    _load().oracle_eri_full(sh, nsh, xyz, ex, co, out)
    return out.reshape(nao, nao, nao, nao)


def schwarz(mol) -> np.ndarray:
    """Q_ab = sqrt(max |(mu nu|mu nu)|) per shell pair (eq:schwartz, shell level)."""
    sh, nsh, xyz, ex, co = _basis_args(mol)
    Q = np.zeros(nsh * nsh)
    _load().oracle_schwarz(sh, nsh, xyz, ex, co, Q)
    return Q.reshape(nsh, nsh)


def schwarz_coulomb(mol) -> np.ndarray:
    """Schwarz factors of the plain 1/r operator, whatever omega is set."""
    lib = _load()
    sh, nsh, xyz, ex, co = _basis_args(mol)
    Q = np.zeros(nsh * nsh)
    # the omega setting is module state of the C library; save, clear, restore
    lib.oracle_set_omega(0.0)
    lib.oracle_schwarz(sh, nsh, xyz, ex, co, Q)
    lib.oracle_set_omega(_current_omega[0])
    return Q.reshape(nsh, nsh)


_current_omega = [0.0]


def dmax(mol, Dcart) -> np.ndarray:
    """Shell-block max |D| over all densities (Cartesian D): the density
    factor of the screening bound of Sec. 2. Pinned against a numpy block
    maximum over two densities, and through the kept quartet counts and the
    restricted-einsum J, K of the screening rule."""
    sh = np.ascontiguousarray(mol.shells, dtype=np.int32)
    nsh = sh.shape[0]
    Dc = np.ascontiguousarray(Dcart, dtype=np.float64)
    ndm, nao = Dc.shape[0], Dc.shape[1]
    out = np.zeros(nsh * nsh)
    _load().oracle_dmax(sh, nsh, Dc.ravel(), ndm, nao, out)
    return out.reshape(nsh, nsh)


# ------------------------------------------------- spherical transform
def _real_solid_harmonic_cart(l: int) -> np.ndarray:
    """C (ncart x (2l+1)): unit-norm real solid harmonics as Cartesian sums.

    Columns m = -l..l, except l = 1 which keeps (x, y, z). Built from the
    closed-form expansion of the real solid harmonics S_lm in Cartesian
    monomials (Schlegel and Frisch, Int. J. Quantum Chem. 54, 83 (1995);
    Helgaker, Jorgensen and Olsen, Sec. 6.4). Pinned: self-overlap identity
    and proportionality to scipy's spherical harmonics.
    """
    comps = cart_components(l)
    if l == 0:
        return np.ones((1, 1))
    if l == 1:
        return np.eye(3)
    C = np.zeros((len(comps), 2 * l + 1))

    def binom(n, k):
        if k < 0 or k > n:
            return 0
        return factorial(n) // (factorial(k) * factorial(n - k))

    for col, m in enumerate(range(-l, l + 1)):
        am = abs(m)
        Nlm = sqrt(2.0 * factorial(l + am) * factorial(l - am) / (1.0 + (m == 0))) / (2 ** am * factorial(l))
        for t in range(0, (l - am) // 2 + 1):
            for u in range(0, t + 1):
                if m >= 0:
                    vs = [v / 2.0 for v in range(0, am + 1, 2)]
                else:
                    vs = [v / 2.0 for v in range(1, am + 1, 2)]
                for v in vs:
                    vm = 0.5 if m < 0 else 0.0
                    coef = ((-1) ** (t + v - vm) * (0.25 ** t) * binom(l, t) * binom(l - t, am + t)
                            * binom(t, u) * binom(am, int(round(2 * v))))
                    lx = int(round(2 * t + am - 2 * (u + v)))
                    ly = int(round(2 * (u + v)))
                    lz = l - lx - ly
                    idx = comps.index((lx, ly, lz))
                    C[idx, col] += Nlm * coef
    # With N_lm above every column has the norm of z^l, i.e. unit norm when
    # the Cartesian (l,0,0) component has unit norm: no rescaling needed.
    return C


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def cart_overlap_one_center(l: int) -> np.ndarray:
    """Overlap of the Cartesian components of one normalised shell with itself.

    For components (lx,ly,lz), (mx,my,mz) of a shell whose (l,0,0) component
    has unit norm: S = prod_k (lk+mk-1)!! / (2l-1)!! when every lk+mk is even,
    else 0 (independent of the exponents and contraction).
    """
    comps = cart_components(l)
    S = np.zeros((len(comps), len(comps)))
    for i, a in enumerate(comps):
        for j, b in enumerate(comps):
            if any((x + y) % 2 for x, y in zip(a, b)):
                continue
            S[i, j] = np.prod([_dfact(x + y - 1) for x, y in zip(a, b)]) / _dfact(2 * l - 1)
    return S


def c2s_matrix(mol) -> np.ndarray:
    """Block-diagonal Cartesian->spherical matrix (nao_cart x nao_sph).

    Shells with spherical == 0 get an identity block.
    """
    blocks = []
    for s in mol.shells:
        l, sph = int(s[1]), int(s[5])
        blocks.append(_real_solid_harmonic_cart(l) if sph else np.eye(ncart(l)))
    ncs = sum(b.shape[0] for b in blocks)
    nss = sum(b.shape[1] for b in blocks)
    C = np.zeros((ncs, nss))
    r = c = 0
    for b in blocks:
        C[r:r + b.shape[0], c:c + b.shape[1]] = b
        r += b.shape[0]
        c += b.shape[1]
    return C


def _to_cart_density(mol, D):
    D = np.asarray(D, dtype=np.float64)
    if D.ndim == 2:
        D = D[None]
    if mol.spherical:
        C = c2s_matrix(mol)
        D = np.stack([C @ d @ C.T for d in D])   # D_cart = C D_sph C^T
    return np.ascontiguousarray(D)


def _from_cart(mol, M):
    if mol.spherical:
        C = c2s_matrix(mol)
        M = np.stack([C.T @ m @ C for m in M])   # X_sph = C^T X_cart C
    return M


# ------------------------------------------------------------ JK builds
def jk(mol, D=None, cutoff: float = 1e-13, with_j=True, with_k=True, use_dmax=True,
       method: str = "screened", Q=None):
    """J and K of eq:jk for ``mol`` (density in the molecule's own basis).

    method = "screened": unique quartets with the 8-fold symmetry and
    degeneracy factors of Sec. 2 (pinned against "brute").
    method = "brute": every shell quartet, no symmetry (plain definition).
    Returns (J, K, nquartets_kept); J/K in the molecule's basis (spherical
    when the shells are spherical).
    """
    lib = _load()
    D = mol.D if D is None else D
    Dc = _to_cart_density(mol, D)
    ndm, nao = Dc.shape[0], Dc.shape[1]
    sh, nsh, xyz, ex, co = _basis_args(mol)
    if Q is None:
        Q = schwarz_coulomb(mol)
    Dm = dmax(mol, Dc)
    J = np.zeros(ndm * nao * nao)
    K = np.zeros(ndm * nao * nao)
    fn = lib.oracle_jk_screened if method == "screened" else lib.oracle_jk_brute
    kept = fn(sh, nsh, xyz, ex, co, np.ascontiguousarray(Q).ravel(), Dm.ravel(), Dc.ravel(),
              ndm, int(bool(with_j)), int(bool(with_k)), float(cutoff), int(bool(use_dmax)), J, K)
    J = _from_cart(mol, J.reshape(ndm, nao, nao))
    K = _from_cart(mol, K.reshape(ndm, nao, nao))
    return J, K, int(kept)


def jk_blocks(mol, jblocks, kblocks, D=None, cutoff: float = 1e-13, with_j=True, with_k=True,
              use_dmax=True, Q=None):
    """Exact Cartesian J blocks (a, b) and K blocks (a, c) straight from eq:jk.

    Cartesian molecules only. Returns (list of J blocks [ndm, na, nb],
    list of K blocks [ndm, na, nc], number of shell quartets evaluated).
    """
    if mol.spherical:
        raise ValueError("jk_blocks works in the Cartesian basis")
    lib = _load()
    D = mol.D if D is None else D
    Dc = _to_cart_density(mol, D)
    ndm, nao = Dc.shape[0], Dc.shape[1]
    sh, nsh, xyz, ex, co = _basis_args(mol)
    if Q is None:
        Q = schwarz_coulomb(mol)
    Dm = dmax(mol, Dc)
    jb = np.ascontiguousarray(np.asarray(jblocks, dtype=np.int32).reshape(-1, 2))
    kb = np.ascontiguousarray(np.asarray(kblocks, dtype=np.int32).reshape(-1, 2))
    ls = sh[:, 1]
    jsz = [ndm * ncart(ls[a]) * ncart(ls[b]) for a, b in jb]
    ksz = [ndm * ncart(ls[a]) * ncart(ls[c]) for a, c in kb]
    jout = np.zeros(max(1, sum(jsz)))
    kout = np.zeros(max(1, sum(ksz)))
    n = lib.oracle_jk_rows(sh, nsh, xyz, ex, co, np.ascontiguousarray(Q).ravel(), Dm.ravel(),
                           Dc.ravel(), ndm, nao, int(bool(with_j)), int(bool(with_k)),
                           float(cutoff), int(bool(use_dmax)),
                           jb.ravel(), len(jb), jout, kb.ravel(), len(kb), kout)
    Jl, Kl = [], []
    o = 0
    for (a, b), s in zip(jb, jsz):
        Jl.append(jout[o:o + s].reshape(ndm, ncart(ls[a]), ncart(ls[b])))
        o += s
    o = 0
    for (a, c), s in zip(kb, ksz):
        Kl.append(kout[o:o + s].reshape(ndm, ncart(ls[a]), ncart(ls[c])))
        o += s
    return Jl, Kl, int(n)


__all__ = ["build", "boys", "eri_prim", "eri_shell", "eri_full", "schwarz", "dmax",
           "jk", "jk_blocks", "c2s_matrix", "cart_overlap_one_center", "cart_components",
           "num_threads", "ncart"]
