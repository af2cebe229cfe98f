"""Pins for the CPU oracle: each checks it against something other than itself.

The paper prints no integral, Boys or J/K values, so the pins are closed
forms, independent quadrature, brute force and the symmetries and bounds of
Sec. 2 (8-fold symmetry, eq:schwartz, eq:jk).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2507_09772_gb300 import synth


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


# ------------------------------------------------------------------ Boys
@pytest.mark.parametrize("m", range(0, 17))
def test_boys_at_zero(m):
    assert oracle.boys(m, 0.0)[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-12, 1e-6, 0.01, 0.5, 3.0, 12.0, 29.99, 30.0, 30.01, 55.0, 400.0])
def test_boys_f0_closed_form(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert oracle.boys(0, T)[0] == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("m,T", [(1, 0.3), (3, 2.5), (6, 9.0), (9, 17.0), (12, 29.5), (12, 30.5),
                                 (4, 45.0), (16, 22.0), (8, 0.001)])
def test_boys_against_adaptive_quadrature(m, T):
    ref, err = integrate.quad(lambda t: t ** (2 * m) * math.exp(-T * t * t), 0.0, 1.0,
                              epsabs=0.0, epsrel=2e-14, limit=200)
    assert oracle.boys(m, T)[m] == pytest.approx(ref, rel=1e-12)


def test_boys_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for m, T in [(0, 7.3), (5, 0.7), (11, 31.0), (14, 60.0), (2, 1e-3)]:
        ref = mp.quad(lambda t: t ** (2 * m) * mp.e ** (-T * t * t), [0, 1])
        assert oracle.boys(m, T)[m] == pytest.approx(float(ref), rel=2e-15)


@pytest.mark.parametrize("m", [0, 1, 4, 8, 12])
def test_boys_large_T_asymptote(m):
    T = 200.0
    asym = _dfact(2 * m - 1) / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
    assert oracle.boys(m, T)[m] == pytest.approx(asym, rel=1e-14)


def test_boys_series_and_recursion_branches_meet():
    # the oracle switches from the series to erf + upward recursion at T = 30;
    # 1e-13 apart, dF_m/dT = -F_{m+1} moves the values by < 1e-13 relative
    lo = oracle.boys(12, 30.0 - 1e-13)
    hi = oracle.boys(12, 30.0 + 1e-13)
    assert np.allclose(lo, hi, rtol=1e-13, atol=0)


# ------------------------------------------------ primitive integrals
def _rng_centers(rng, spread=1.5):
    return rng.uniform(-spread, spread, size=(4, 3))


def test_ssss_closed_form():
    rng = np.random.default_rng(7)
    for _ in range(20):
        al = np.exp(rng.uniform(np.log(0.05), np.log(300.0), size=4))
        R = _rng_centers(rng)
        a, b, c, d = al
        p, q = a + b, c + d
        P = (a * R[0] + b * R[1]) / p
        Q = (c * R[2] + d * R[3]) / q
        Kab = math.exp(-a * b / p * np.sum((R[0] - R[1]) ** 2))
        Kcd = math.exp(-c * d / q * np.sum((R[2] - R[3]) ** 2))
        T = p * q / (p + q) * np.sum((P - Q) ** 2)
        F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * F0
        val = oracle.eri_prim((0, 0, 0, 0), al, R)[0, 0, 0, 0]
        assert val == pytest.approx(ref, rel=1e-14)


def _richardson_derivative(f, x0, h):
    d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
    d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("center", [0, 1, 2, 3])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("lbase", [0, 1, 2, 3])
def test_centre_derivative_raises_angular_momentum(center, axis, lbase):
    """x-power raising from a centre derivative, on every centre and axis.

    For phi = (x-A_x)^k ... exp(-alpha |r-A|^2):
        d phi / d A_x = -k phi[k-1] + 2 alpha phi[k+1],
    so phi[k+1] = (d phi/d A_x + k phi[k-1]) / (2 alpha). Checked with a
    Richardson-extrapolated central difference of the oracle's own blocks
    at the lower angular momentum.
    """
    rng = np.random.default_rng(100 + 12 * center + 3 * axis + lbase)
    al = np.exp(rng.uniform(np.log(0.3), np.log(4.0), size=4))
    R0 = _rng_centers(rng, 1.2)
    ls = [1, 0, 1, 0]
    ls[center] = lbase
    hi = list(ls)
    hi[center] = lbase + 1
    blk_hi = oracle.eri_prim(hi, al, R0)
    comps_lo = oracle.cart_components(lbase)
    comps_hi = oracle.cart_components(lbase + 1)

    def block_at(shift):
        R = R0.copy()
        R[center, axis] += shift
        return oracle.eri_prim(ls, al, R)

    dblk = _richardson_derivative(block_at, 0.0, 1e-3)
    lo_blk = oracle.eri_prim(ls, al, R0)
    lower = oracle.eri_prim([x - 1 if i == center else x for i, x in enumerate(ls)], al, R0) \
        if lbase > 0 else None
    comps_lower = oracle.cart_components(lbase - 1) if lbase > 0 else []
    alpha = al[center]
    checked = 0
    for j, cmp in enumerate(comps_lo):
        up = list(cmp)
        up[axis] += 1
        k = cmp[axis]
        ih = comps_hi.index(tuple(up))
        pred = np.take(dblk, j, axis=center)
        if k > 0:
            dn = list(cmp)
            dn[axis] -= 1
            pred = pred + k * np.take(lower, comps_lower.index(tuple(dn)), axis=center)
        pred = pred / (2 * alpha)
        got = np.take(blk_hi, ih, axis=center)
        scale = max(1e-3, np.abs(got).max())
        assert np.abs(got - pred).max() < 2e-8 * scale
        checked += 1
    assert checked == len(comps_lo)
    del lo_blk


# ----------------- independent Gaussian-transform quadrature of (ab|cd)
_GH_X, _GH_W = np.polynomial.hermite.hermgauss(24)


def _pair_1d_tables(u, la, lb, lc, ld, a, b, c, d, A, B, C, D):
    """G[ax,bx,cx,dx] = integral over x1, x2 of
    (x1-A)^ax (x1-B)^bx exp(-a(x1-A)^2 - b(x1-B)^2) exp(-u^2 (x1-x2)^2)
    (x2-C)^cx (x2-D)^dx exp(-c(x2-C)^2 - d(x2-D)^2),
    by a 2D Gauss-Hermite rule after diagonalising the quadratic form."""
    p, q = a + b, c + d
    P = (a * A + b * B) / p
    Q = (c * C + d * D) / q
    pre = math.exp(-a * b / p * (A - B) ** 2 - c * d / q * (C - D) ** 2)
    u2 = u * u
    M = np.array([[p + u2, -u2], [-u2, q + u2]])
    w = u2 * (P - Q) * np.array([1.0, -1.0])
    z0 = -np.linalg.solve(M, w)
    const = u2 * (P - Q) ** 2 + w @ z0
    L = np.linalg.cholesky(M)
    Linv_T = np.linalg.inv(L).T
    y1, y2 = np.meshgrid(_GH_X, _GH_X, indexing="ij")
    wt = np.outer(_GH_W, _GH_W)
    Y = np.stack([y1.ravel(), y2.ravel()])
    Z = z0[:, None] + Linv_T @ Y
    x1 = Z[0] + P
    x2 = Z[1] + Q
    jac = 1.0 / np.prod(np.diag(L))
    base = wt.ravel() * jac * pre * math.exp(-const)
    out = np.zeros((la + 1, lb + 1, lc + 1, ld + 1))
    pa = np.stack([(x1 - A) ** k for k in range(la + 1)])
    pb = np.stack([(x1 - B) ** k for k in range(lb + 1)])
    pc = np.stack([(x2 - C) ** k for k in range(lc + 1)])
    pd = np.stack([(x2 - D) ** k for k in range(ld + 1)])
    out = np.einsum("in,jn,kn,ln,n->ijkl", pa, pb, pc, pd, base)
    return out


def quadrature_eri(ls, al, R, u_lo=0.0, u_hi=None):
    """Gaussian-transform quadrature of (ab|cd) for the operator
    (2/sqrt(pi)) int_{u_lo}^{u_hi} exp(-u^2 r^2) du: 1/r for [0, inf),
    erf(w r)/r for [0, w], erfc(w r)/r for [w, inf)."""
    la, lb, lc, ld = ls
    ca, cb, cc, cd = (oracle.cart_components(l) for l in ls)

    def integrand(u):
        G = [_pair_1d_tables(u, la, lb, lc, ld, *al, R[0, k], R[1, k], R[2, k], R[3, k])
             for k in range(3)]
        blk = np.empty((len(ca), len(cb), len(cc), len(cd)))
        for i, A_ in enumerate(ca):
            for j, B_ in enumerate(cb):
                for k, C_ in enumerate(cc):
                    for l, D_ in enumerate(cd):
                        v = 1.0
                        for x in range(3):
                            v *= G[x][A_[x], B_[x], C_[x], D_[x]]
                        blk[i, j, k, l] = v
        return blk.ravel()

    # 1/r12 = (2/sqrt(pi)) int_0^inf exp(-u^2 r12^2) du; map u = u_lo + s/(1-s)
    if u_hi is None:
        def mapped(s):
            u = u_lo + s / (1.0 - s)
            return integrand(u) / (1.0 - s) ** 2
        val, err = integrate.quad_vec(mapped, 0.0, 1.0, epsabs=1e-14, epsrel=1e-11, limit=400)
    else:
        val, err = integrate.quad_vec(integrand, u_lo, u_hi, epsabs=1e-14, epsrel=1e-11, limit=400)
    return 2.0 / math.sqrt(math.pi) * val.reshape(len(ca), len(cb), len(cc), len(cd))


@pytest.mark.parametrize("ls", [(1, 0, 0, 0), (1, 1, 0, 0), (0, 0, 1, 1), (1, 0, 1, 0),
                                (2, 0, 1, 0), (2, 1, 0, 1), (2, 2, 0, 0), (2, 0, 2, 0),
                                (3, 0, 1, 0), (1, 2, 2, 1), (3, 1, 2, 0), (2, 2, 2, 2),
                                (4, 0, 1, 0), (2, 1, 4, 0)])
def test_eri_against_gaussian_transform_quadrature(ls):
    rng = np.random.default_rng(sum(l * 7 ** i for i, l in enumerate(ls)))
    al = np.exp(rng.uniform(np.log(0.2), np.log(3.0), size=4))
    R = _rng_centers(rng, 1.0)
    ref = quadrature_eri(ls, al, R)
    got = oracle.eri_prim(ls, al, R)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() < 1e-10 * scale


# ----------------------------------------------- tensor-level structure
@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_631gs()


@pytest.fixture(scope="module")
def tiny_eri(tiny):
    return oracle.eri_full(tiny)


def test_eightfold_symmetry(tiny_eri):
    g = tiny_eri
    s = np.abs(g).max()
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0), (2, 3, 1, 0)]:
        assert np.abs(g - g.transpose(perm)).max() < 1e-14 * s


def test_schwarz_inequality_elementwise(tiny_eri):
    g = tiny_eri
    n = g.shape[0]
    diag = np.einsum("ijij->ij", g)
    assert (diag >= -1e-14).all()
    bound = np.sqrt(np.maximum(diag, 0.0)).reshape(n * n)
    lhs = np.abs(g.reshape(n * n, n * n))
    assert (lhs <= np.outer(bound, bound) * (1 + 1e-12) + 1e-15).all()


def test_schwarz_table_matches_full_tensor(tiny, tiny_eri):
    Q = oracle.schwarz(tiny)
    off = np.cumsum([0] + [oracle.ncart(int(l)) for l in tiny.shells[:, 1]])
    diag = np.einsum("ijij->ij", tiny_eri)
    for a in range(tiny.nshell):
        for b in range(tiny.nshell):
            blk = diag[off[a]:off[a + 1], off[b]:off[b + 1]]
            assert Q[a, b] == pytest.approx(math.sqrt(np.abs(blk).max()), rel=1e-14)


def test_jk_equals_einsum_of_full_tensor(tiny, tiny_eri):
    D = tiny.D[0]
    Jref = np.einsum("ijkl,kl->ij", tiny_eri, D)
    Kref = np.einsum("ijkl,jl->ik", tiny_eri, D)
    J, K, _ = oracle.jk(tiny, cutoff=0.0, method="brute")
    assert np.abs(J[0] - Jref).max() < 1e-12
    assert np.abs(K[0] - Kref).max() < 1e-12
    J2, K2, _ = oracle.jk(tiny, cutoff=0.0, method="screened")
    assert np.abs(J2[0] - Jref).max() < 1e-12
    assert np.abs(K2[0] - Kref).max() < 1e-12


def test_screened_symmetric_equals_brute_force(tiny):
    for cutoff in (1e-13, 1e-8, 1e-4):
        for wj, wk in ((1, 1), (1, 0), (0, 1)):
            J1, K1, n1 = oracle.jk(tiny, cutoff=cutoff, with_j=wj, with_k=wk, method="brute")
            J2, K2, n2 = oracle.jk(tiny, cutoff=cutoff, with_j=wj, with_k=wk, method="screened")
            assert np.abs(J1 - J2).max() < 1e-13
            assert np.abs(K1 - K2).max() < 1e-13
            assert n2 <= n1


def test_jk_symmetric_and_positive(tiny):
    J, K, _ = oracle.jk(tiny)
    assert np.abs(J - J.transpose(0, 2, 1)).max() < 1e-13
    assert np.abs(K - K.transpose(0, 2, 1)).max() < 1e-13
    D = tiny.D[0]
    assert np.einsum("ij,ij->", D, J[0]) > 0
    assert np.einsum("ij,ij->", D, K[0]) > 0


def test_two_densities_are_independent(tiny):
    rng = np.random.default_rng(3)
    D2 = synth.random_density(rng, tiny.nao, 7, 1)[0]
    Dboth = np.stack([tiny.D[0], D2])
    J, K, _ = oracle.jk(tiny, D=Dboth)
    J1, K1, _ = oracle.jk(tiny, D=Dboth[:1])
    # screening uses the max over both densities, so compare with a cutoff of 0
    J, K, _ = oracle.jk(tiny, D=Dboth, cutoff=0.0)
    J1, K1, _ = oracle.jk(tiny, D=Dboth[:1], cutoff=0.0)
    J2, K2, _ = oracle.jk(tiny, D=Dboth[1:], cutoff=0.0)
    assert np.abs(J[0] - J1[0]).max() < 1e-13 and np.abs(J[1] - J2[0]).max() < 1e-13
    assert np.abs(K[0] - K1[0]).max() < 1e-13 and np.abs(K[1] - K2[0]).max() < 1e-13


def test_translation_invariance(tiny):
    J, K, _ = oracle.jk(tiny)
    moved = synth.Molecule(coords=tiny.coords + np.array([3.1, -7.2, 0.4]), shells=tiny.shells,
                           exps=tiny.exps, coeffs=tiny.coeffs, nao=tiny.nao,
                           nao_cart=tiny.nao_cart, D=tiny.D)
    J2, K2, _ = oracle.jk(moved)
    assert np.abs(J - J2).max() < 1e-12
    assert np.abs(K - K2).max() < 1e-12


def test_axis_relabelling_permutes_components(tiny):
    """New frame (x', y', z') = (y, z, x): component (lx,ly,lz) of the new
    frame is component (lz,lx,ly) of the old one."""
    perm = []
    for s in tiny.shells:
        l, ao = int(s[1]), int(s[4])
        comps = oracle.cart_components(l)
        for (lx, ly, lz) in comps:
            perm.append(ao + comps.index((lz, lx, ly)))
    perm = np.array(perm)
    D = tiny.D[0]
    Dn = D[np.ix_(perm, perm)][None]
    moved = synth.Molecule(coords=tiny.coords[:, [1, 2, 0]].copy(), shells=tiny.shells,
                           exps=tiny.exps, coeffs=tiny.coeffs, nao=tiny.nao,
                           nao_cart=tiny.nao_cart, D=Dn)
    J, K, _ = oracle.jk(tiny, cutoff=0.0)
    Jn, Kn, _ = oracle.jk(moved, cutoff=0.0)
    assert np.abs(Jn[0] - J[0][np.ix_(perm, perm)]).max() < 1e-12
    assert np.abs(Kn[0] - K[0][np.ix_(perm, perm)]).max() < 1e-12


def test_row_blocks_match_full_build(tiny):
    J, K, _ = oracle.jk(tiny)
    off = np.cumsum([0] + [oracle.ncart(int(l)) for l in tiny.shells[:, 1]])
    rng = np.random.default_rng(5)
    jb = rng.integers(0, tiny.nshell, size=(6, 2))
    kb = rng.integers(0, tiny.nshell, size=(6, 2))
    Jl, Kl, _ = oracle.jk_blocks(tiny, jb, kb)
    for (a, b), blk in zip(jb, Jl):
        assert np.abs(blk[0] - J[0][off[a]:off[a + 1], off[b]:off[b + 1]]).max() < 1e-12
    for (a, c), blk in zip(kb, Kl):
        assert np.abs(blk[0] - K[0][off[a]:off[a + 1], off[c]:off[c + 1]]).max() < 1e-12


def test_normalised_basis_diagonal_integral_of_tight_s_shell():
    """A single normalised s primitive: (ss|ss) = 2 sqrt(2 alpha/pi)... for one
    centre, (aa|aa) = 2 pi^{5/2}/(p^2 sqrt(2p)) N^4 with p = 2 alpha and
    N = (2 alpha/pi)^{3/4}, which is sqrt(4 alpha/pi)."""
    for alpha in (0.1, 1.0, 37.0, 5000.0):
        rng = np.random.default_rng(0)
        mol = synth.custom_basis_molecule(np.zeros((1, 3)), [[(0, [alpha])]], rng, nocc=1)
        v = oracle.eri_shell(mol, 0, 0, 0, 0)[0, 0, 0, 0]
        assert v == pytest.approx(math.sqrt(4 * alpha / math.pi), rel=1e-14)


# ------------------------------------------------------------ spherical
@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_spherical_self_overlap_is_identity(l):
    mol_like = synth.Molecule(coords=np.zeros((1, 3)),
                              shells=np.array([[0, l, 1, 0, 0, 1]], dtype=np.int32),
                              exps=np.ones(1), coeffs=np.ones(1), nao=2 * l + 1,
                              nao_cart=oracle.ncart(l))
    C = oracle.c2s_matrix(mol_like)
    S = oracle.cart_overlap_one_center(l)
    assert np.abs(C.T @ S @ C - np.eye(2 * l + 1)).max() < 1e-14


@pytest.mark.parametrize("l", [2, 3, 4])
def test_spherical_columns_are_real_spherical_harmonics(l):
    from scipy import special
    rng = np.random.default_rng(l)
    v = rng.standard_normal((40, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    theta = np.arccos(v[:, 2])
    phi = np.arctan2(v[:, 1], v[:, 0])
    mol_like = synth.Molecule(coords=np.zeros((1, 3)),
                              shells=np.array([[0, l, 1, 0, 0, 1]], dtype=np.int32),
                              exps=np.ones(1), coeffs=np.ones(1), nao=2 * l + 1,
                              nao_cart=oracle.ncart(l))
    C = oracle.c2s_matrix(mol_like)
    comps = oracle.cart_components(l)
    mono = np.stack([v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c for a, b, c in comps], axis=1)
    S = mono @ C

    def Y(m):
        if hasattr(special, "sph_harm_y"):
            y = special.sph_harm_y(l, abs(m), theta, phi)
        else:
            y = special.sph_harm(abs(m), l, phi, theta)
        if m > 0:
            return np.sqrt(2) * y.real
        if m < 0:
            return np.sqrt(2) * y.imag
        return y.real

    for col, m in enumerate(range(-l, l + 1)):
        ratio = S[:, col] / Y(m)
        assert np.std(ratio) < 1e-10 * np.abs(ratio).mean()


def test_spherical_trace_identity():
    mol = synth.random_small_molecule(11, natm=2, lmax=3, max_nprim=2, spherical=True)
    J, K, _ = oracle.jk(mol, cutoff=0.0)
    C = oracle.c2s_matrix(mol)
    Dc = np.einsum("ip,pq,jq->ij", C, mol.D[0], C)
    cart = synth.Molecule(coords=mol.coords, shells=mol.shells * np.array([1, 1, 1, 1, 1, 0]),
                          exps=mol.exps, coeffs=mol.coeffs, nao=mol.nao_cart,
                          nao_cart=mol.nao_cart, D=Dc[None])
    Jc, Kc, _ = oracle.jk(cart, cutoff=0.0)
    assert np.einsum("ij,ij->", mol.D[0], J[0]) == pytest.approx(np.einsum("ij,ij->", Dc, Jc[0]),
                                                                  rel=1e-12)
    assert np.einsum("ij,ij->", mol.D[0], K[0]) == pytest.approx(np.einsum("ij,ij->", Dc, Kc[0]),
                                                                  rel=1e-12)


# ------------------------------------------------- range-separated Coulomb
@pytest.mark.parametrize("omega", [0.2, 0.7, 3.0])
def test_long_range_ssss_closed_form(omega):
    rng = np.random.default_rng(int(omega * 10))
    for _ in range(10):
        al = np.exp(rng.uniform(np.log(0.05), np.log(50.0), size=4))
        R = _rng_centers(rng)
        a, b, c, d = al
        p, q = a + b, c + d
        P = (a * R[0] + b * R[1]) / p
        Q = (c * R[2] + d * R[3]) / q
        Kab = math.exp(-a * b / p * np.sum((R[0] - R[1]) ** 2))
        Kcd = math.exp(-c * d / q * np.sum((R[2] - R[3]) ** 2))
        rho = p * q / (p + q)
        theta = omega ** 2 / (omega ** 2 + rho)
        T = theta * rho * np.sum((P - Q) ** 2)
        F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * math.sqrt(theta) * F0
        with oracle.omega_operator(omega):
            val = oracle.eri_prim((0, 0, 0, 0), al, R)[0, 0, 0, 0]
        assert val == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("ls", [(1, 0, 0, 0), (1, 1, 1, 0), (2, 1, 0, 1), (2, 2, 1, 1)])
@pytest.mark.parametrize("omega", [0.4, -0.4, 1.5, -1.5])
def test_range_separated_against_quadrature(ls, omega):
    rng = np.random.default_rng(sum(ls) + int(abs(omega) * 10))
    al = np.exp(rng.uniform(np.log(0.2), np.log(3.0), size=4))
    R = _rng_centers(rng, 1.0)
    w = abs(omega)
    ref = quadrature_eri(ls, al, R, 0.0, w) if omega > 0 else quadrature_eri(ls, al, R, w, None)
    with oracle.omega_operator(omega):
        got = oracle.eri_prim(ls, al, R)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def test_long_range_tends_to_full_coulomb():
    rng = np.random.default_rng(3)
    al = np.exp(rng.uniform(np.log(0.2), np.log(3.0), size=4))
    R = _rng_centers(rng, 1.0)
    full = oracle.eri_prim((2, 1, 1, 0), al, R)
    with oracle.omega_operator(1e6):
        lr = oracle.eri_prim((2, 1, 1, 0), al, R)
    assert np.abs(lr - full).max() < 1e-9 * np.abs(full).max()


def test_range_separated_jk_is_symmetric_and_ordered():
    mol = synth.tiny_631gs()
    Jf, Kf, _ = oracle.jk(mol, cutoff=0.0)
    with oracle.omega_operator(0.3):
        Jl, Kl, _ = oracle.jk(mol, cutoff=0.0)
    with oracle.omega_operator(-0.3):
        Js, Ks, _ = oracle.jk(mol, cutoff=0.0)
    assert np.abs(Jl + Js - Jf).max() < 1e-12
    assert np.abs(Kl + Ks - Kf).max() < 1e-12
    D = mol.D[0]
    # both attenuated operators are positive definite
    for J in (Jl, Js):
        assert np.einsum("ij,ij->", D, J[0]) > 0


def test_g_shell_molecule_screened_equals_brute_force_and_einsum():
    """With g shells (l = 4): the symmetric screened builder equals the
    brute-force builder over every shell quartet and the einsum of the full
    ERI tensor, and J, K stay symmetric with tr(DJ), tr(DK) >= 0."""
    rng = np.random.default_rng(404)
    xyz = np.array([[0.0, 0.0, 0.0], [1.2, 0.4, -0.3]])
    per_atom = [[(0, [2.5, 0.4]), (4, [0.9])], [(1, [0.7]), (4, [1.3])]]
    mol = synth.custom_basis_molecule(xyz, per_atom, rng, name="g-pin")
    J1, K1, _ = oracle.jk(mol, cutoff=0.0, method="brute")
    J2, K2, _ = oracle.jk(mol, cutoff=0.0, method="screened")
    assert np.abs(J1 - J2).max() < 1e-12 * max(1.0, np.abs(J1).max())
    assert np.abs(K1 - K2).max() < 1e-12 * max(1.0, np.abs(K1).max())
    eri = oracle.eri_full(mol)
    D = mol.D[0]
    Je = np.einsum("ijkl,kl->ij", eri, D)
    Ke = np.einsum("ijkl,jl->ik", eri, D)
    assert np.abs(J2[0] - Je).max() < 1e-12 * max(1.0, np.abs(Je).max())
    assert np.abs(K2[0] - Ke).max() < 1e-12 * max(1.0, np.abs(Ke).max())
    assert np.abs(J2[0] - J2[0].T).max() < 1e-13 and np.abs(K2[0] - K2[0].T).max() < 1e-13
    assert np.trace(D @ J2[0]) >= 0 and np.trace(D @ K2[0]) >= 0


# ------------------------------------------- density maxima and screening
# The screening rule of Sec. 2 (eq:schwartz times the density bound): a shell
# quartet (ab|cd) is kept iff Q_ab Q_cd Dmax > cutoff, with Dmax the largest
# |D| over every density in the blocks the requested outputs read (ab, cd for
# J; ac, ad, bc, bd for K). These pins restate the block maximum and the rule
# in numpy, independently of the C code, and check (1) the block maxima
# exactly, (2) the kept counts exactly, (3) J and K equal to the einsum of the
# full ERI tensor restricted to the kept quartets, and (4) the error against
# the unscreened einsum within the Schwarz bound of the dropped quartets.
def _shell_offsets(mol):
    return np.cumsum([0] + [oracle.ncart(int(l)) for l in mol.shells[:, 1]])


def _np_block_max(mol, Dcart):
    off = _shell_offsets(mol)
    A = np.abs(Dcart).max(axis=0)
    n = mol.nshell
    out = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            out[a, b] = A[off[a]:off[a + 1], off[b]:off[b + 1]].max()
    return out


def _np_schwarz_from_tensor(mol, eri):
    off = _shell_offsets(mol)
    diag = np.abs(np.einsum("ijij->ij", eri))
    n = mol.nshell
    Q = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            Q[a, b] = math.sqrt(diag[off[a]:off[a + 1], off[b]:off[b + 1]].max())
    return Q


def _np_kept(Q, Dm, cutoff, with_j, with_k):
    """Kept mask over every ordered shell quartet (a, b, c, d)."""
    n = Q.shape[0]
    dm = np.zeros((n, n, n, n))
    if with_j:
        dm = np.maximum(dm, Dm[:, :, None, None])
        dm = np.maximum(dm, Dm[None, None, :, :])
    if with_k:
        dm = np.maximum(dm, Dm[:, None, :, None])   # ac
        dm = np.maximum(dm, Dm[:, None, None, :])   # ad
        dm = np.maximum(dm, Dm[None, :, :, None])   # bc
        dm = np.maximum(dm, Dm[None, :, None, :])   # bd
    # the same product order as the rule states it: (Q_ab Q_cd) Dmax
    B = (Q[:, :, None, None] * Q[None, None, :, :]) * dm
    return B > cutoff


def _n_unique(mask):
    n = mask.shape[0]
    cnt = 0
    for a in range(n):
        for b in range(a + 1):
            for c in range(n):
                for d in range(c + 1):
                    if a * (a + 1) // 2 + b >= c * (c + 1) // 2 + d and mask[a, b, c, d]:
                        cnt += 1
    return cnt


def _g_screen_molecule():
    """Two atoms 3 Å apart with s, p and g shells (tight and diffuse), so
    that the rule drops a good share of the quartets at 1e-8 and 1e-4."""
    rng = np.random.default_rng(404)
    xyz = np.array([[0.0, 0.0, 0.0], [3.0, 0.4, -0.3]])
    per_atom = [[(0, [2.5, 0.4]), (4, [0.9]), (0, [8.0])], [(1, [0.7]), (4, [1.3]), (0, [6.0])]]
    return synth.custom_basis_molecule(xyz, per_atom, rng, name="g-screen")


def _two_densities(mol, seed):
    """D1 the molecule's own density; D2 a symmetric random matrix whose
    elements are scaled so that each density holds the largest element of
    some shell blocks."""
    rng = np.random.default_rng(seed)
    D1 = mol.D[0]
    R = rng.standard_normal(D1.shape) * np.exp(rng.uniform(-3.0, 1.0, size=D1.shape))
    D2 = 0.5 * np.abs(D1).max() * (R + R.T) / np.abs(R + R.T).max()
    return np.stack([D1, D2])


def test_density_block_max_matches_numpy_over_two_densities(tiny):
    Dboth = _two_densities(tiny, 11)
    got = oracle.dmax(tiny, Dboth)
    ref = _np_block_max(tiny, Dboth)
    assert np.array_equal(got, ref)
    # both densities decide some blocks, and blocks of every l pair occur
    m1 = _np_block_max(tiny, Dboth[:1])
    m2 = _np_block_max(tiny, Dboth[1:])
    assert (m1 > m2).any() and (m2 > m1).any()
    assert len({(int(tiny.shells[a, 1]), int(tiny.shells[b, 1]))
                for a in range(tiny.nshell) for b in range(tiny.nshell)}) == 9


@pytest.fixture(scope="module")
def screening_cases(tiny, tiny_eri):
    g = _g_screen_molecule()
    return [("tiny", tiny, tiny_eri, _two_densities(tiny, 12)),
            ("g-screen", g, oracle.eri_full(g), _two_densities(g, 13))]


@pytest.mark.parametrize("cutoff", [1e-8, 1e-4])
@pytest.mark.parametrize("with_j,with_k", [(1, 1), (1, 0), (0, 1)])
def test_screening_rule_kept_set_and_result(screening_cases, cutoff, with_j, with_k):
    for name, mol, eri, D in screening_cases:
        Q = _np_schwarz_from_tensor(mol, eri)
        Dm = _np_block_max(mol, D)
        mask = _np_kept(Q, Dm, cutoff, with_j, with_k)
        assert 0 < mask.sum() < mask.size, name   # the rule drops something and keeps something
        J1, K1, n1 = oracle.jk(mol, D=D, cutoff=cutoff, with_j=with_j, with_k=with_k, method="brute", Q=Q)
        J2, K2, n2 = oracle.jk(mol, D=D, cutoff=cutoff, with_j=with_j, with_k=with_k, method="screened", Q=Q)
        assert n1 == int(mask.sum()), name
        assert n2 == _n_unique(mask), name
        off = _shell_offsets(mol)
        sh_of = np.repeat(np.arange(mol.nshell), np.diff(off))
        M = mask[np.ix_(sh_of, sh_of, sh_of, sh_of)]
        kept = eri * M
        scale = max(1.0, np.abs(eri).max() * np.abs(D).max() * mol.nao ** 2)
        for m in range(D.shape[0]):
            if with_j:
                Jm = np.einsum("ijkl,kl->ij", kept, D[m])
                assert np.abs(J1[m] - Jm).max() < 1e-13 * scale, name
                assert np.abs(J2[m] - Jm).max() < 1e-13 * scale, name
            if with_k:
                Km = np.einsum("ijkl,jl->ik", kept, D[m])
                assert np.abs(K1[m] - Km).max() < 1e-13 * scale, name
                assert np.abs(K2[m] - Km).max() < 1e-13 * scale, name


@pytest.mark.parametrize("cutoff", [1e-8, 1e-4])
@pytest.mark.parametrize("with_j,with_k", [(1, 1), (1, 0), (0, 1)])
def test_screening_error_within_schwarz_bound_of_dropped_quartets(screening_cases, cutoff, with_j, with_k):
    """|J - J_full| and |K - K_full| (J_full, K_full: einsum of the whole ERI
    tensor) are at most the sum, over the quartets the rule drops, of
    Q_ab Q_cd max|D in the contracted block| times the block size (eq:schwartz
    bounds every element of a block by Q_ab Q_cd)."""
    for name, mol, eri, D in screening_cases:
        Q = _np_schwarz_from_tensor(mol, eri)
        Dm = _np_block_max(mol, D)
        drop = ~_np_kept(Q, Dm, cutoff, with_j, with_k)
        assert drop.any(), name
        off = _shell_offsets(mol)
        nf = np.diff(off).astype(float)
        sh_of = np.repeat(np.arange(mol.nshell), nf.astype(int))
        J, K, _ = oracle.jk(mol, D=D, cutoff=cutoff, with_j=with_j, with_k=with_k, method="screened", Q=Q)
        QQ = Q[:, :, None, None] * Q[None, None, :, :] * drop
        # J_ab element: sum over dropped (c, d) of Q_ab Q_cd max|D_cd| N_c N_d
        jb = np.einsum("abcd,cd->ab", QQ, Dm * np.outer(nf, nf))
        # K_ac element: sum over dropped (b, d) of Q_ab Q_cd max|D_bd| N_b N_d
        kb = np.einsum("abcd,bd->ac", QQ, Dm * np.outer(nf, nf))
        Jb = jb[np.ix_(sh_of, sh_of)]
        Kb = kb[np.ix_(sh_of, sh_of)]
        for m in range(D.shape[0]):
            if with_j:
                Jf = np.einsum("ijkl,kl->ij", eri, D[m])
                err = np.abs(J[m] - Jf)
                # plus rounding of the sums themselves
                assert (err <= Jb * (1 + 1e-12) + 1e-13 * max(1.0, np.abs(Jf).max())).all(), name
            if with_k:
                Kf = np.einsum("ijkl,jl->ik", eri, D[m])
                err = np.abs(K[m] - Kf)
                assert (err <= Kb * (1 + 1e-12) + 1e-13 * max(1.0, np.abs(Kf).max())).all(), name
        # and the rule is not vacuous: at 1e-4 the dropped quartets matter
        if cutoff == 1e-4 and with_j:
            Jf = np.einsum("ijkl,kl->ij", eri, D[0])
            assert np.abs(J[0] - Jf).max() > 1e-9, name
