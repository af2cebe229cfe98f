"""Seeded synthetic molecules, basis sets and density matrices.

This module only draws inputs. It holds none of the JK method's arithmetic
(no integrals, no Boys function, no screening): both the CUDA path and the
CPU oracle consume what it returns, and neither is imported here.

Shapes follow the workloads the paper benchmarks on (Sec. 3.1 and 3.2: a
6-31G*-sized basis with s/p/d shells and contractions up to 6, and a
def2-TZVPP-sized basis with shells up to f and contractions up to 8). The
real molecules and the public basis-set files are not used; every value
below is a seeded draw.

Conventions shared by every consumer of these arrays
----------------------------------------------------
* Coordinates are in bohr (1 angstrom = 1/0.529177210903 bohr).
* A shell record is ``(atom, l, nprim, prim_off, ao_off, spherical)``.
  ``ao_off`` counts Cartesian functions when ``spherical == 0`` and real
  solid harmonics (2l+1 per shell) when ``spherical == 1``.
* Cartesian components of a shell are ordered with the x exponent
  descending, then y descending (xx, xy, xz, yy, yz, zz for d), the
  ordering of Sec. 2.
* ``coeffs[prim_off + i]`` multiplies the *unnormalised* primitive
  ``x^lx y^ly z^lz exp(-exps[prim_off + i] r^2)``. The value folds in the
  primitive normalisation of the (l,0,0) component and a contraction
  normalisation that gives the contracted (l,0,0) component unit norm.
  Other Cartesian components keep their natural norms.
* Densities are ``D = C C^T`` with ``C`` the Q factor of a QR of a standard
  normal (nao x nocc) matrix, so D is symmetric and positive semidefinite.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import pi

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903

# (l, nprim) per shell, in the order the shells are laid out on an atom.
HEAVY_631GS = [(0, 6), (0, 3), (0, 1), (1, 3), (1, 1), (2, 1)]
LIGHT_631GS_P = [(0, 3), (0, 1), (1, 1)]        # light atom of the batched workload
LIGHT_631GS = [(0, 3), (0, 1)]                  # light atom of the large clusters
HEAVY_TZVPP = [(0, 8), (0, 2), (0, 1), (0, 1), (0, 1),
               (1, 4), (1, 1), (1, 1), (2, 1), (2, 1), (3, 1)]
LIGHT_TZVPP = [(0, 3), (0, 1), (0, 1), (1, 1), (1, 1), (2, 1)]

SHELL_RECORD = ("atom", "l", "nprim", "prim_off", "ao_off", "spherical")


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nsph(l: int) -> int:
    return 2 * l + 1


@dataclass
class Molecule:
    """One molecule: basis arrays in the layout ``jk_init`` takes, plus D."""
    coords: np.ndarray            # (natm, 3) float64, bohr
    shells: np.ndarray            # (nshell, 6) int32, see SHELL_RECORD
    exps: np.ndarray              # (nprim_total,) float64
    coeffs: np.ndarray            # (nprim_total,) float64, normalised
    nao: int                      # functions in the basis D is given in
    nao_cart: int                 # Cartesian functions
    D: np.ndarray | None = None   # (n_dm, nao, nao) float64
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def natm(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shells.shape[0])

    @property
    def spherical(self) -> bool:
        return bool(self.shells[:, 5].any()) if self.nshell else False


# --------------------------------------------------------------------------
# normalisation of the (l,0,0) component (input convention, not the method)
# --------------------------------------------------------------------------
def _dfact(n: int) -> int:
    """(n)!! with (-1)!! = 0!! = 1."""
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def _gauss_x2l_integral(l: int, a: float) -> float:
    """Integral over R^3 of x^(2l) exp(-a r^2)."""
    return _dfact(2 * l - 1) / (2.0 * a) ** l * (pi / a) ** 1.5


def normalised_coefficients(l: int, exps: np.ndarray, raw: np.ndarray) -> np.ndarray:
    """Fold primitive and contraction normalisation into ``raw``."""
    exps = np.asarray(exps, dtype=np.float64)
    c = np.asarray(raw, dtype=np.float64).copy()
    for i, a in enumerate(exps):
        c[i] /= np.sqrt(_gauss_x2l_integral(l, 2.0 * a))
    s = 0.0
    for i, a in enumerate(exps):
        for j, b in enumerate(exps):
            s += c[i] * c[j] * _gauss_x2l_integral(l, a + b)
    return c / np.sqrt(s)


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------
def _rejection_box(rng, n: int, side_ang: float, min_sep_ang: float, max_tries=200000):
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rejection sampling did not converge")
        x = rng.uniform(0.0, side_ang, size=3)
        if all(np.linalg.norm(x - p) >= min_sep_ang for p in pts):
            pts.append(x)
    return np.array(pts)


def _rejection_sphere(rng, n: int, radius_ang: float, min_sep_ang: float, max_tries=200000):
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rejection sampling did not converge")
        x = rng.uniform(-radius_ang, radius_ang, size=3)
        if np.linalg.norm(x) > radius_ang:
            continue
        if all(np.linalg.norm(x - p) >= min_sep_ang for p in pts):
            pts.append(x)
    return np.array(pts)


def _random_rotation(rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# --------------------------------------------------------------------------
# per-atom exponent ladders
# --------------------------------------------------------------------------
def _ladder_assign(template, ladders, rng):
    """Exponent arrays per shell of one atom.

    ``ladders[l]`` is a geometric series that the shells of angular momentum
    ``l`` take rungs from in order; ``None`` draws log-uniform in a range.
    """
    out = []
    used = {}
    for l, npr in template:
        lad = ladders[l]
        if isinstance(lad, tuple) and lad[0] == "loguniform":
            lo, hi = lad[1], lad[2]
            out.append(np.exp(rng.uniform(np.log(lo), np.log(hi), size=npr)))
            continue
        k = used.get(l, 0)
        out.append(np.asarray(lad[k:k + npr], dtype=np.float64))
        used[l] = k + npr
    return out


def _atom_exponents(kind: str, rng):
    if kind == "heavy631":
        tpl = HEAVY_631GS
        lad = {0: np.geomspace(5000.0, 0.1, 10), 1: np.geomspace(50.0, 0.1, 4),
               2: ("loguniform", 0.4, 1.2)}
    elif kind == "light631p":
        tpl = LIGHT_631GS_P
        lad = {0: np.geomspace(30.0, 0.1, 4), 1: ("loguniform", 0.5, 1.5)}
    elif kind == "light631":
        tpl = LIGHT_631GS
        lad = {0: np.geomspace(30.0, 0.1, 4)}
    elif kind == "heavytz":
        tpl = HEAVY_TZVPP
        lad = {0: np.geomspace(3.0e4, 0.05, 13), 1: np.geomspace(60.0, 0.08, 6),
               2: np.geomspace(2.5, 0.25, 2), 3: ("loguniform", 0.8, 1.6)}
    elif kind == "lighttz":
        tpl = LIGHT_TZVPP
        lad = {0: np.geomspace(35.0, 0.05, 5), 1: np.geomspace(1.5, 0.4, 2),
               2: ("loguniform", 0.8, 1.3)}
    else:
        raise ValueError(kind)
    exps = _ladder_assign(tpl, lad, rng)
    scale = np.exp(rng.uniform(-0.1, 0.1))
    return tpl, [e * scale for e in exps]


def build_molecule(coords_ang: np.ndarray, kinds, rng, spherical: bool = False,
                   name: str = "") -> Molecule:
    """Assemble the basis arrays for atoms of the given kinds."""
    shells, exps, coeffs = [], [], []
    ao = 0
    ao_cart = 0
    pofs = 0
    for ia, kind in enumerate(kinds):
        tpl, ex = _atom_exponents(kind, rng)
        for (l, npr), e in zip(tpl, ex):
            raw = rng.uniform(0.1, 1.0, size=npr)
            c = normalised_coefficients(l, e, raw)
            shells.append((ia, l, npr, pofs, ao, 1 if spherical else 0))
            exps.extend(e.tolist())
            coeffs.extend(c.tolist())
            pofs += npr
            ao += nsph(l) if spherical else ncart(l)
            ao_cart += ncart(l)
    return Molecule(coords=np.asarray(coords_ang, dtype=np.float64) * BOHR_PER_ANGSTROM,
                    shells=np.asarray(shells, dtype=np.int32).reshape(-1, 6),
                    exps=np.asarray(exps, dtype=np.float64),
                    coeffs=np.asarray(coeffs, dtype=np.float64),
                    nao=ao, nao_cart=ao_cart, name=name)


def random_density(rng, nao: int, nocc: int, n_dm: int = 1) -> np.ndarray:
    """D = C C^T with C the orthonormal Q factor of a Gaussian matrix."""
    out = np.empty((n_dm, nao, nao))
    for k in range(n_dm):
        q, _ = np.linalg.qr(rng.standard_normal((nao, nocc)))
        out[k] = q @ q.T
    return out


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def tiny_631gs(seed: int = 1000, n_dm: int = 1) -> Molecule:
    """3 heavy atoms in a 3 A cube, 45 Cartesian functions, nocc = 11."""
    rng = np.random.default_rng(seed)
    xyz = _rejection_box(rng, 3, 3.0, 0.9)
    mol = build_molecule(xyz, ["heavy631"] * 3, rng, name="tiny-631gs")
    mol.D = random_density(rng, mol.nao, 11, n_dm)
    return mol


def batched_molecule(m: int, seed_base: int = 1001, n_dm: int = 1,
                     natm: int | None = None) -> Molecule:
    """Molecule ``m`` of the batched workload: 10-60 atoms, 2:1 light:heavy."""
    rng = np.random.default_rng(seed_base + m)
    n = int(rng.integers(10, 61)) if natm is None else int(natm)
    nheavy = int(round(n / 3))
    kinds = ["heavy631"] * nheavy + ["light631p"] * (n - nheavy)
    rng.shuffle(kinds)
    side = (n / 0.1) ** (1.0 / 3.0)
    xyz = _rejection_box(rng, n, side, 0.9)
    mol = build_molecule(xyz, kinds, rng, name=f"batch-{m}")
    mol.D = random_density(rng, mol.nao, mol.nao // 4, n_dm)
    mol.meta["natm"] = n
    return mol


def batched_631gs(nmol: int = 64, seed_base: int = 1001, n_dm: int = 1):
    """64 independent molecules of 10-60 atoms (the batched workload)."""
    return [batched_molecule(m, seed_base, n_dm) for m in range(nmol)]


def _triatomic_cluster(rng, nunits: int, extra_light: int = 0):
    spacing = 0.0334 ** (-1.0 / 3.0)
    nside = int(np.ceil(nunits ** (1.0 / 3.0) - 1e-9))
    sites = np.array([(i, j, k) for i in range(nside) for j in range(nside)
                      for k in range(nside)], dtype=np.float64) * spacing
    pick = rng.choice(len(sites), size=nunits, replace=False)
    centres = []
    for s in sites[pick]:
        for _ in range(1000):
            c = s + rng.uniform(-0.3, 0.3, size=3)
            if all(np.linalg.norm(c - p) >= 2.4 for p in centres):
                centres.append(c)
                break
        else:
            raise RuntimeError("could not place unit")
    half = np.deg2rad(104.5) / 2.0
    xyz, kinds = [], []
    for c in centres:
        rot = _random_rotation(rng)
        r1 = 1.0 + rng.uniform(-0.05, 0.05)
        r2 = 1.0 + rng.uniform(-0.05, 0.05)
        v1 = rot @ np.array([np.sin(half), 0.0, np.cos(half)]) * r1
        v2 = rot @ np.array([-np.sin(half), 0.0, np.cos(half)]) * r2
        xyz += [c, c + v1, c + v2]
        kinds += ["heavy631", "light631", "light631"]
    free = [i for i in range(len(sites)) if i not in set(pick.tolist())]
    for _ in range(extra_light):
        s = sites[free[int(rng.integers(len(free)))]]
        xyz.append(s + rng.uniform(-0.3, 0.3, size=3))
        kinds.append("light631")
    return np.array(xyz), kinds


def water_like_cluster(nunits: int = 256, seed: int = 1002, n_dm: int = 1,
                       extra_light: int = 0) -> Molecule:
    """Triatomic units at liquid-water number density (mixed-precision workload)."""
    rng = np.random.default_rng(seed)
    xyz, kinds = _triatomic_cluster(rng, nunits, extra_light)
    mol = build_molecule(xyz, kinds, rng, name=f"cluster-{len(kinds)}")
    mol.D = random_density(rng, mol.nao, mol.nao // 4, n_dm)
    return mol


def router_cluster(seed: int = 1004, n_dm: int = 1) -> Molecule:
    """1,024 atoms: 341 triatomic units plus one extra light atom."""
    return water_like_cluster(341, seed, n_dm, extra_light=1)


def highl_tzvpp(seed: int = 1003, n_dm: int = 1, spherical: bool = True) -> Molecule:
    """60-atom globular cluster (20 heavy, 40 light) with a TZVPP-shaped basis."""
    rng = np.random.default_rng(seed)
    radius = (60 / 0.1 * 3.0 / (4.0 * pi)) ** (1.0 / 3.0)
    xyz = _rejection_sphere(rng, 60, radius, 0.9)
    kinds = ["heavytz"] * 20 + ["lighttz"] * 40
    rng.shuffle(kinds)
    mol = build_molecule(xyz, kinds, rng, spherical=spherical, name="highl-tzvpp")
    mol.D = random_density(rng, mol.nao, mol.nao // 4, n_dm)
    return mol


def custom_basis_molecule(coords_ang, shells_per_atom, rng, spherical=False,
                          nocc=None, n_dm=1, name="custom") -> Molecule:
    """Any atoms with an explicit list of (l, exps) per atom (micro-benchmarks)."""
    shells, exps, coeffs = [], [], []
    ao = ao_cart = pofs = 0
    for ia, lst in enumerate(shells_per_atom):
        for l, e in lst:
            e = np.atleast_1d(np.asarray(e, dtype=np.float64))
            raw = rng.uniform(0.1, 1.0, size=len(e))
            c = normalised_coefficients(l, e, raw)
            shells.append((ia, l, len(e), pofs, ao, 1 if spherical else 0))
            exps.extend(e.tolist())
            coeffs.extend(c.tolist())
            pofs += len(e)
            ao += nsph(l) if spherical else ncart(l)
            ao_cart += ncart(l)
    mol = Molecule(coords=np.asarray(coords_ang, dtype=np.float64) * BOHR_PER_ANGSTROM,
                   shells=np.asarray(shells, dtype=np.int32).reshape(-1, 6),
                   exps=np.asarray(exps), coeffs=np.asarray(coeffs),
                   nao=ao, nao_cart=ao_cart, name=name)
    if nocc is None:
        nocc = max(1, mol.nao // 4)
    mol.D = random_density(rng, mol.nao, nocc, n_dm)
    return mol


def random_small_molecule(seed: int, natm: int = 2, lmax: int = 2, max_nprim: int = 3,
                          n_dm: int = 1, spherical: bool = False) -> Molecule:
    """Small random test molecule with every angular momentum up to ``lmax``."""
    rng = np.random.default_rng(seed)
    xyz = _rejection_box(rng, natm, 2.5, 0.8)
    per_atom = []
    for _ in range(natm):
        lst = []
        for l in range(lmax + 1):
            npr = int(rng.integers(1, max_nprim + 1))
            e = np.sort(np.exp(rng.uniform(np.log(0.15), np.log(40.0), size=npr)))[::-1]
            lst.append((l, e))
        per_atom.append(lst)
    return custom_basis_molecule(xyz, per_atom, rng, spherical=spherical,
                                 n_dm=n_dm, name=f"rand-{seed}")


def workload(name: str, **kw):
    """Named workloads: tiny, batch, cluster, highl, router."""
    if name == "tiny":
        return tiny_631gs(**kw)
    if name == "batch":
        return batched_631gs(**kw)
    if name == "cluster":
        return water_like_cluster(**kw)
    if name == "highl":
        return highl_tzvpp(**kw)
    if name == "router":
        return router_cluster(**kw)
    raise ValueError(name)


__all__ = [
    "Molecule", "BOHR_PER_ANGSTROM", "ncart", "nsph", "normalised_coefficients",
    "build_molecule", "random_density", "tiny_631gs", "batched_molecule",
    "batched_631gs", "water_like_cluster", "router_cluster", "highl_tzvpp",
    "custom_basis_molecule", "random_small_molecule", "workload",
]
