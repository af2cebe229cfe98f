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
