"""Parity at full workload sizes, in the launch configuration bench.py times.

The oracle cannot build J and K of these systems whole in seconds, so it
computes sampled shell blocks one by one (oracle.jk_blocks: J_ab and K_ac
straight from eq:jk over every screened quartet) and the GPU result is
compared on those blocks.
"""
import numpy as np
import pytest

import oracle
from paper_2507_09772_gb300 import jk, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    jk.load_library()


def _blocks(mol, rng, nj, nk):
    ns = mol.nshell
    jb = np.stack([rng.integers(0, ns, nj), rng.integers(0, ns, nj)], axis=1)
    kb = np.stack([rng.integers(0, ns, nk), rng.integers(0, ns, nk)], axis=1)
    return jb, kb


def _compare(mol, J, K, jb, kb, tol):
    off = np.cumsum([0] + [oracle.ncart(int(l)) for l in mol.shells[:, 1]])
    Jl, Kl, _ = oracle.jk_blocks(mol, jb, kb, cutoff=1e-13)
    for (a, b), blk in zip(jb, Jl):
        g = J[0][off[a]:off[a + 1], off[b]:off[b + 1]]
        assert np.abs(g - blk[0]).max() <= tol, ("J", a, b)
    for (a, c), blk in zip(kb, Kl):
        g = K[0][off[a]:off[a + 1], off[c]:off[c + 1]]
        assert np.abs(g - blk[0]).max() <= tol, ("K", a, c)


@pytest.fixture(scope="module")
def batched():
    """The 64-molecule benchmark batch, built as bench.py builds it."""
    mols = synth.batched_631gs(64)
    eng = jk.JK(mols)
    eng.set_option("use_graph", 1)
    eng.set_option("branches", 4)
    Ds = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in mols]
    J, K, st = eng.build(Ds, cutoff=1e-13, stats=True)
    Jm, Km, stm = eng.build(Ds, cutoff=1e-13, precision="mixed", stats=True)
    torch.cuda.synchronize()
    out = (mols, [j.cpu().numpy() for j in J], [k.cpu().numpy() for k in K],
           [j.cpu().numpy() for j in Jm], [k.cpu().numpy() for k in Km], st, stm)
    eng.close()
    return out


def test_batched_workload_fp64_sampled_blocks(batched):
    mols, J, K, _, _, st, _ = batched
    rng = np.random.default_rng(0)
    order = sorted(range(len(mols)), key=lambda i: mols[i].natm)
    for i in (order[0], order[len(order) // 2], order[-1]):   # smallest, median, largest
        jb, kb = _blocks(mols[i], rng, 4, 3)
        _compare(mols[i], J[i], K[i], jb, kb, TOL64)


def test_batched_workload_mixed_against_fp64_everywhere(batched):
    mols, J, K, Jm, Km, st, stm = batched
    assert stm["quartets_fp64"] + stm["quartets_fp32"] == st["quartets_fp64"]
    assert max(np.abs(a - b).max() for a, b in zip(J, Jm)) <= TOL_MIXED
    assert max(np.abs(a - b).max() for a, b in zip(K, Km)) <= TOL_MIXED


def test_highl_cluster_cartesian_sampled_blocks():
    """60-atom TZVPP-shaped cluster (f shells, 8-primitive core s), Cartesian."""
    mol = synth.highl_tzvpp(spherical=False)
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J, K, st = eng.build(D, cutoff=1e-13, stats=True)
    torch.cuda.synchronize()
    eng.close()
    rng = np.random.default_rng(1)
    jb, kb = _blocks(mol, rng, 2, 2)
    _compare(mol, J.cpu().numpy(), K.cpu().numpy(), jb, kb, TOL64)


def _near_and_random_pairs(mol, rng, n_near, n_rand, lmax=4):
    """Shell pairs: n_near with both shells within 2.5 bohr (large Q_ab, the
    blocks that carry most of J), n_rand uniform; shells of l <= lmax (the
    oracle's cost of a block grows steeply with its angular momenta)."""
    ok = np.nonzero(mol.shells[:, 1] <= lmax)[0]
    xyz = np.asarray(mol.coords)[mol.shells[:, 0]]
    out = []
    while len(out) < n_near:
        a = int(rng.choice(ok))
        near = ok[np.linalg.norm(xyz[ok] - xyz[a], axis=1) < 2.5]
        out.append((a, int(rng.choice(near))))
    for _ in range(n_rand):
        out.append((int(rng.choice(ok)), int(rng.choice(ok))))
    return np.array(out, dtype=np.int64)


def test_water_cluster_fp64_and_mixed_sampled_blocks():
    """768-atom water-like cluster (4,864 functions, the mixed-precision
    workload): FP64 and mixed builds in the launch configuration bench.py
    times, against 8 J and 8 K oracle blocks at 1e-10 (FP64) and 1e-8
    (mixed); the mixed build evaluates every quartet the FP64 build does,
    most of them in FP32."""
    mol = synth.water_like_cluster()
    assert mol.natm == 768 and mol.nao == 4864
    eng = jk.JK(mol)
    eng.set_option("use_graph", 1)
    eng.set_option("branches", 4)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J, K, st = eng.build(D, cutoff=1e-13, stats=True)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    Jm, Km, stm = eng.build(D, cutoff=1e-13, precision="mixed", stats=True)
    Jm, Km = Jm.cpu().numpy(), Km.cpu().numpy()
    eng.close()
    assert stm["quartets_fp64"] + stm["quartets_fp32"] == st["quartets_fp64"]
    assert stm["quartets_fp32"] > 0.5 * st["quartets_fp64"]
    rng = np.random.default_rng(2)
    jb = _near_and_random_pairs(mol, rng, 4, 4)
    kb = _near_and_random_pairs(mol, rng, 4, 4)
    off = np.cumsum([0] + [oracle.ncart(int(l)) for l in mol.shells[:, 1]])
    Jl, Kl, _ = oracle.jk_blocks(mol, jb, kb, cutoff=1e-13)
    assert max(np.abs(b).max() for b in Jl) > 1e-2   # blocks that carry J
    for (a, b), blk in zip(jb, Jl):
        sl = (slice(off[a], off[a + 1]), slice(off[b], off[b + 1]))
        assert np.abs(J[0][sl] - blk[0]).max() <= TOL64, ("J", a, b)
        assert np.abs(Jm[0][sl] - blk[0]).max() <= TOL_MIXED, ("J mixed", a, b)
    for (a, c), blk in zip(kb, Kl):
        sl = (slice(off[a], off[a + 1]), slice(off[c], off[c + 1]))
        assert np.abs(K[0][sl] - blk[0]).max() <= TOL64, ("K", a, c)
        assert np.abs(Km[0][sl] - blk[0]).max() <= TOL_MIXED, ("K mixed", a, c)
    # everywhere: the mixed build against the FP64 build
    assert np.abs(Jm - J).max() <= TOL_MIXED and np.abs(Km - K).max() <= TOL_MIXED


def test_highl_cluster_spherical_mixed_sampled_blocks():
    """60-atom TZVPP-shaped cluster in its spherical basis (1,180 functions),
    mixed precision: J_sph and K_sph blocks against C_a^T X_cart C_b from the
    oracle's Cartesian blocks of D_cart = C D_sph C^T, at 1e-8."""
    mol = synth.highl_tzvpp(spherical=True)
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J, K, st = eng.build(D, cutoff=1e-13, precision="mixed", stats=True)
    torch.cuda.synchronize()
    eng.close()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    assert st["quartets_fp32"] > 0 and st["quartets_fp64"] > 0
    C = oracle.c2s_matrix(mol)
    cart = synth.Molecule(coords=mol.coords, shells=mol.shells.copy(), exps=mol.exps, coeffs=mol.coeffs,
                          nao=mol.nao_cart, nao_cart=mol.nao_cart, name="highl-cart")
    cart.shells[:, 5] = 0
    Dc = np.stack([C @ d @ C.T for d in mol.D])   # D_cart = C D_sph C^T
    rng = np.random.default_rng(3)
    jb = _near_and_random_pairs(cart, rng, 1, 1, lmax=1)
    kb = _near_and_random_pairs(cart, rng, 1, 1, lmax=1)
    Jl, Kl, _ = oracle.jk_blocks(cart, jb, kb, D=Dc, cutoff=1e-13)
    offc = np.cumsum([0] + [oracle.ncart(int(l)) for l in mol.shells[:, 1]])
    offs = np.cumsum([0] + [2 * int(l) + 1 for l in mol.shells[:, 1]])
    for blocks, vals, X in ((jb, Jl, J), (kb, Kl, K)):
        for (a, b), blk in zip(blocks, vals):
            Ca = C[offc[a]:offc[a + 1], offs[a]:offs[a + 1]]
            Cb = C[offc[b]:offc[b + 1], offs[b]:offs[b + 1]]
            ref = Ca.T @ blk[0] @ Cb
            got = X[0][offs[a]:offs[a + 1], offs[b]:offs[b + 1]]
            assert np.abs(got - ref).max() <= TOL_MIXED, (a, b)
