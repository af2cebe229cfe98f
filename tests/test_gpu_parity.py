"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: max |dJ|, |dK| <= 1e-10 for all-FP64 builds and <= 1e-8 for
mixed precision (the bounds the JK method is held to); the FP32-only mode is
checked against a looser bound derived from single precision.
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


def gpu_jk(mol, D=None, **kw):
    eng = jk.JK(mol)
    try:
        for k, v in kw.pop("options", {}).items():
            eng.set_option(k, v)
        Dn = mol.D if D is None else D
        Dt = torch.tensor(np.asarray(Dn), dtype=torch.float64, device="cuda")
        J, K, st = eng.build(Dt, stats=True, **kw)
        torch.cuda.synchronize()
        return (None if J is None else J.cpu().numpy(), None if K is None else K.cpu().numpy(), st)
    finally:
        eng.close()


def maxdiff(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def where_wrong(mol, A, B, tol):
    """Shell blocks (l, nprim) of the largest mismatches, for failure messages."""
    d = np.abs(np.asarray(A) - np.asarray(B))
    if d.ndim == 3:
        d = d.max(axis=0)
    off = np.cumsum([0] + [oracle.ncart(int(l)) for l in mol.shells[:, 1]])
    sh_of = np.searchsorted(off, np.arange(off[-1]), side="right") - 1
    bad = {}
    for i, j in zip(*np.nonzero(d > tol)):
        a, b = sh_of[i], sh_of[j]
        key = (int(mol.shells[a, 1]), int(mol.shells[a, 2]), int(mol.shells[b, 1]), int(mol.shells[b, 2]))
        bad[key] = max(bad.get(key, 0.0), float(d[i, j]))
    return sorted(bad.items(), key=lambda kv: -kv[1])[:8]


def check(mol, got, ref, tol, what):
    err = maxdiff(got, ref)
    assert err <= tol, f"{what}: max err {err:.3e}; worst blocks (la,na,lb,nb): {where_wrong(mol, got, ref, tol)}"


def test_tiny_fp64_matches_oracle():
    mol = synth.tiny_631gs()
    J, K, st = gpu_jk(mol, cutoff=1e-13, precision="fp64")
    Jr, Kr, nq = oracle.jk(mol, cutoff=1e-13)
    check(mol, J, Jr, TOL64, "J")
    check(mol, K, Kr, TOL64, "K")
    assert abs(st["quartets_fp64"] - nq) <= 2
    assert st["quartets_fp32"] == 0


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_random_molecules_fp64(seed):
    mol = synth.random_small_molecule(seed, natm=2 + seed % 2, lmax=2, max_nprim=3)
    J, K, _ = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    check(mol, J, Jr, TOL64, "J")
    check(mol, K, Kr, TOL64, "K")


def test_ten_atom_molecule_spans_many_ket_chunks():
    mol = synth.batched_molecule(0, natm=10)
    J, K, st = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, nq = oracle.jk(mol, cutoff=1e-13)
    assert maxdiff(J, Jr) <= TOL64
    assert maxdiff(K, Kr) <= TOL64
    assert abs(st["quartets_fp64"] - nq) <= max(2, nq // 100000)


def test_two_densities():
    mol = synth.tiny_631gs(n_dm=2)
    J, K, _ = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    assert J.shape == (2, mol.nao, mol.nao)
    assert maxdiff(J, Jr) <= TOL64
    assert maxdiff(K, Kr) <= TOL64


@pytest.mark.parametrize("wj,wk", [(1, 0), (0, 1)])
def test_j_only_and_k_only(wj, wk):
    mol = synth.tiny_631gs()
    J, K, _ = gpu_jk(mol, cutoff=1e-13, with_j=bool(wj), with_k=bool(wk))
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13, with_j=wj, with_k=wk)
    if wj:
        assert maxdiff(J, Jr) <= TOL64 and K is None
    if wk:
        assert maxdiff(K, Kr) <= TOL64 and J is None


@pytest.mark.parametrize("cutoff", [0.0, 1e-10, 1e-6])
def test_cutoffs(cutoff):
    mol = synth.tiny_631gs()
    J, K, st = gpu_jk(mol, cutoff=cutoff)
    Jr, Kr, nq = oracle.jk(mol, cutoff=cutoff)
    assert maxdiff(J, Jr) <= TOL64
    assert maxdiff(K, Kr) <= TOL64
    if cutoff > 0:
        assert abs(st["quartets_fp64"] - nq) <= 2
    else:
        # the library drops shell pairs with Q_ab <= pair_cutoff (1e-18) at init,
        # the oracle keeps every quartet with a bound above 0
        Q = oracle.schwarz(mol)
        iu = np.tril_indices(mol.nshell)
        q = Q[iu]
        npair_kept = int((q > 1e-18).sum())
        assert st["quartets_fp64"] == npair_kept * (npair_kept + 1) // 2


def test_schwarz_factors_match_oracle():
    mol = synth.tiny_631gs()
    eng = jk.JK(mol)
    Q = jk.jk_schwarz(eng.h)
    eng.close()
    Qr = oracle.schwarz(mol)
    kept = Qr > 1e-18
    assert np.allclose(Q[kept], Qr[kept], rtol=1e-12, atol=0)
    assert np.all(Q[~kept] == 0.0)   # pairs at or below pair_cutoff are dropped at init


def test_without_density_screening():
    mol = synth.tiny_631gs()
    J, K, _ = gpu_jk(mol, cutoff=1e-11, options={"use_dmax": 0})
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-11, use_dmax=False)
    assert maxdiff(J, Jr) <= TOL64
    assert maxdiff(K, Kr) <= TOL64


def test_single_s_shell_and_single_d_shell():
    rng = np.random.default_rng(0)
    for lst in ([[(0, [1.3])]], [[(2, [0.8])]], [[(1, [2.0, 0.5])], [(0, [0.7])]]):
        mol = synth.custom_basis_molecule(rng.uniform(0, 1.5, size=(len(lst), 3)), lst, rng, nocc=1)
        J, K, _ = gpu_jk(mol, cutoff=0.0)
        Jr, Kr, _ = oracle.jk(mol, cutoff=0.0)
        assert maxdiff(J, Jr) <= TOL64 and maxdiff(K, Kr) <= TOL64


def test_batch_matches_per_molecule_oracle():
    mols = [synth.random_small_molecule(20 + i, natm=2, lmax=2, max_nprim=2) for i in range(3)]
    mols.append(synth.tiny_631gs())
    eng = jk.JK(mols)
    Ds = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in mols]
    J, K, st = eng.build(Ds, cutoff=1e-13, stats=True)
    torch.cuda.synchronize()
    eng.close()
    total = 0
    for m, j, k in zip(mols, J, K):
        Jr, Kr, nq = oracle.jk(m, cutoff=1e-13)
        total += nq
        assert maxdiff(j.cpu().numpy(), Jr) <= TOL64
        assert maxdiff(k.cpu().numpy(), Kr) <= TOL64
    assert abs(st["quartets_fp64"] - total) <= 4


def test_repeated_builds_are_reproducible_to_atomic_reordering():
    mol = synth.batched_molecule(1, natm=10)
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J1, K1, _ = eng.build(D)
    J2, K2, _ = eng.build(D)
    torch.cuda.synchronize()
    eng.close()
    assert float((J1 - J2).abs().max()) <= 1e-12
    assert float((K1 - K2).abs().max()) <= 1e-12


def test_mixed_precision_within_tolerance():
    mol = synth.batched_molecule(2, natm=12)
    J, K, st = gpu_jk(mol, cutoff=1e-13, precision="mixed")
    Jr, Kr, nq = oracle.jk(mol, cutoff=1e-13)
    assert st["quartets_fp32"] > 0 and st["quartets_fp64"] > 0
    assert maxdiff(J, Jr) <= TOL_MIXED
    assert maxdiff(K, Kr) <= TOL_MIXED


@pytest.mark.parametrize("opts", [{"asym64": 1}, {"screen64": 0}, {"widen_int": 1}, {"chunk_fp64tier": 64}])
def test_mixed_precision_options_within_tolerance(opts):
    """The precision and scheduling options of a mixed build (FP64 large-T
    Rys limit, plain FP32 bound compares, integer widening, FP64-tier work
    items) against the oracle; every option keeps each quartet in exactly
    one tier, so the quartet counts match the FP64 build (plain FP32
    compares may flip a quartet within one rounding of the cutoff)."""
    mol = synth.batched_molecule(2, natm=12)
    _, _, s64 = gpu_jk(mol, cutoff=1e-13)
    J, K, st = gpu_jk(mol, cutoff=1e-13, precision="mixed", options=opts)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    assert st["quartets_fp32"] > 0 and st["quartets_fp64"] > 0
    flips = max(4, int(1e-6 * s64["quartets_fp64"])) if "screen64" in opts else 0
    assert abs(st["quartets_fp64"] + st["quartets_fp32"] - s64["quartets_fp64"]) <= flips
    assert maxdiff(J, Jr) <= TOL_MIXED
    assert maxdiff(K, Kr) <= TOL_MIXED


def test_fp32_mode_error_is_single_precision_sized():
    mol = synth.tiny_631gs()
    J, K, st = gpu_jk(mol, cutoff=1e-13, precision="fp32")
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    assert st["quartets_fp64"] == 0
    scale = max(np.abs(Jr).max(), 1.0)
    assert maxdiff(J, Jr) <= 1e-4 * scale
    assert maxdiff(K, Kr) <= 1e-4 * scale


def test_bad_arguments_return_codes():
    mol = synth.tiny_631gs()
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    lib = jk.load_library()
    assert lib.jk_build(eng.h, D.data_ptr(), 0, 1, 1, 1e-13, 0, J.data_ptr(), K.data_ptr(), None, None) == jk.JK_ERR_ARG
    assert lib.jk_build(eng.h, D.data_ptr(), 9, 1, 1, 1e-13, 0, J.data_ptr(), K.data_ptr(), None, None) == jk.JK_ERR_UNSUPPORTED
    assert lib.jk_build(eng.h, D.data_ptr(), 1, 0, 0, 1e-13, 0, J.data_ptr(), K.data_ptr(), None, None) == jk.JK_ERR_ARG
    assert lib.jk_build(eng.h, D.data_ptr(), 1, 1, 1, -1.0, 0, J.data_ptr(), K.data_ptr(), None, None) == jk.JK_ERR_ARG
    assert lib.jk_build(eng.h, D.data_ptr(), 1, 1, 1, 1e-13, 7, J.data_ptr(), K.data_ptr(), None, None) == jk.JK_ERR_ARG
    assert lib.jk_build(eng.h, None, 1, 1, 1, 1e-13, 0, J.data_ptr(), K.data_ptr(), None, None) == jk.JK_ERR_ARG
    # the handle still works afterwards
    J2, K2, _ = eng.build(D)
    torch.cuda.synchronize()
    eng.close()
    Jr, Kr, _ = oracle.jk(mol)
    assert maxdiff(J2.cpu().numpy(), Jr) <= TOL64


@pytest.mark.parametrize("seed", [31, 32])
def test_spherical_d_molecules(seed):
    mol = synth.random_small_molecule(seed, natm=2, lmax=2, max_nprim=2, spherical=True)
    J, K, _ = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    assert J.shape == (1, mol.nao, mol.nao)
    assert maxdiff(J, Jr) <= TOL64
    assert maxdiff(K, Kr) <= TOL64


@pytest.mark.parametrize("spherical", [False, True])
def test_f_shells(spherical):
    mol = synth.random_small_molecule(41, natm=2, lmax=3, max_nprim=2, spherical=spherical)
    J, K, _ = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    check(mol, J, Jr, TOL64, "J")
    check(mol, K, Kr, TOL64, "K")


def test_tzvpp_shaped_pair_of_atoms():
    rng = np.random.default_rng(7)
    xyz = np.array([[0.0, 0.0, 0.0], [1.1, 0.3, -0.4]])
    mol = synth.build_molecule(xyz, ["heavytz", "lighttz"], rng, spherical=True)
    mol.D = synth.random_density(rng, mol.nao, mol.nao // 4)
    J, K, _ = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    assert maxdiff(J, Jr) <= TOL64
    assert maxdiff(K, Kr) <= TOL64


@pytest.mark.parametrize("branches", [1, 4])
def test_graph_replay_and_branches_match_eager(branches):
    mols = [synth.batched_molecule(3, natm=10), synth.tiny_631gs()]
    eng = jk.JK(mols)
    Ds = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in mols]
    J0, K0, s0 = eng.build(Ds, stats=True)
    eng.set_option("use_graph", 1)
    eng.set_option("branches", branches)
    J1, K1, s1 = eng.build(Ds, stats=True)          # captures
    Ds2 = [d.clone() for d in Ds]                    # new buffers: descriptors change, graph reused
    J2, K2, s2 = eng.build(Ds2, stats=True)
    torch.cuda.synchronize()
    assert eng.get_option("graphs") == 1
    eng.close()
    for a, b, c in zip(J0, J1, J2):
        assert float((a - b).abs().max()) <= 1e-12 and float((a - c).abs().max()) <= 1e-12
    for a, b, c in zip(K0, K1, K2):
        assert float((a - b).abs().max()) <= 1e-12 and float((a - c).abs().max()) <= 1e-12
    assert s0["quartets_fp64"] == s1["quartets_fp64"] == s2["quartets_fp64"]


def test_partitioned_builds_sum_to_the_full_build():
    mols = [synth.batched_molecule(8, natm=12), synth.tiny_631gs()]
    eng = jk.JK(mols)
    Ds = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in mols]
    J0, K0, s0 = eng.build(Ds, stats=True)
    Js = [torch.zeros_like(d) for d in Ds]
    Ks = [torch.zeros_like(d) for d in Ds]
    nq = 0
    eng.set_option("part_count", 3)
    for p in range(3):
        eng.set_option("part_index", p)
        J, K, st = eng.build(Ds, stats=True)
        nq += st["quartets_fp64"]
        for a, b in zip(Js, J):
            a += b
        for a, b in zip(Ks, K):
            a += b
    torch.cuda.synchronize()
    eng.close()
    assert nq == s0["quartets_fp64"]
    for a, b in zip(Js, J0):
        assert float((a - b).abs().max()) <= 1e-12
    for a, b in zip(Ks, K0):
        assert float((a - b).abs().max()) <= 1e-12


def test_primitive_screening_changes_nothing_beyond_its_threshold():
    mol = synth.batched_molecule(9, natm=14)
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J1, K1, s1 = eng.build(D, stats=True)                 # default: prim_eps = 1e-16
    eng.set_option("prim_eps", 0.0)
    J0, K0, s0 = eng.build(D, stats=True)                 # every primitive quartet
    torch.cuda.synchronize()
    eng.close()
    assert s1["quartets_fp64"] == s0["quartets_fp64"]
    assert s1["prim_quartets"] < s0["prim_quartets"]
    assert float((J1 - J0).abs().max()) <= 1e-12
    assert float((K1 - K0).abs().max()) <= 1e-12


@pytest.mark.parametrize("omega", [0.3, -0.3, 2.0])
def test_range_separated_operators_match_oracle(omega):
    mol = synth.random_small_molecule(51, natm=2, lmax=2, max_nprim=2)
    J, K, _ = gpu_jk(mol, cutoff=1e-13, options={"omega": omega})
    with oracle.omega_operator(omega):
        Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    check(mol, J, Jr, TOL64, "J")
    check(mol, K, Kr, TOL64, "K")


def test_long_plus_short_range_is_coulomb():
    mol = synth.tiny_631gs()
    Jf, Kf, _ = gpu_jk(mol, cutoff=1e-13)
    Jl, Kl, _ = gpu_jk(mol, cutoff=1e-13, options={"omega": 0.4})
    Js, Ks, _ = gpu_jk(mol, cutoff=1e-13, options={"omega": -0.4})
    assert np.abs(Jl + Js - Jf).max() <= 1e-11
    assert np.abs(Kl + Ks - Kf).max() <= 1e-11


def test_incremental_density_build_screens_on_the_change():
    """Direct-SCF incremental build (Sec. 2, density screening with Delta D):
    J(D2) = J(D1) + J(D2 - D1), the increment screened by |D2 - D1|."""
    mol = synth.batched_molecule(10, natm=12)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((mol.nao, mol.nao)) * 1e-8   # a late-SCF-sized change
    D1 = mol.D
    D2 = D1 + (X + X.T)[None]
    J1, K1, s1 = gpu_jk(mol, D=D1, cutoff=1e-13)
    Jd, Kd, sd = gpu_jk(mol, D=D2 - D1, cutoff=1e-13)
    J2, K2, s2 = gpu_jk(mol, D=D2, cutoff=1e-13)
    assert np.abs(J1 + Jd - J2).max() <= 1e-10
    assert np.abs(K1 + Kd - K2).max() <= 1e-10
    # the increment itself against the oracle, screened the same way by
    # |Delta D| (the values are ~1e-8, so the bound is far below TOL64; a
    # quartet within rounding of the cutoff changes J or K by < 1e-13 N_f^2)
    Jr, Kr, nr = oracle.jk(mol, D=D2 - D1, cutoff=1e-13)
    assert np.abs(Jd - Jr).max() <= 1e-11 and np.abs(Kd - Kr).max() <= 1e-11
    assert np.abs(Jd).max() > 1e-9   # the comparison is not vacuous
    assert abs(sd["quartets_fp64"] - nr) <= max(2, 1e-4 * nr)
    # a random density does not decay with distance, so most of the 12-atom
    # molecule's quartets stay above 1e-13 even at |Delta D| ~ 1e-8
    assert sd["quartets_fp64"] < 0.75 * s2["quartets_fp64"]


def test_separate_j_and_k_builds_screen_on_their_own_blocks():
    mol = synth.batched_molecule(11, natm=16)
    _, _, sjk = gpu_jk(mol, cutoff=1e-13)
    J, _, sj = gpu_jk(mol, cutoff=1e-13, with_k=False)
    _, K, sk = gpu_jk(mol, cutoff=1e-13, with_j=False)
    assert sj["quartets_fp64"] <= sjk["quartets_fp64"] and sk["quartets_fp64"] <= sjk["quartets_fp64"]
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13, with_k=False)
    assert np.abs(J - Jr).max() <= TOL64
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13, with_j=False)
    assert np.abs(K - Kr).max() <= TOL64


def test_non_finite_density_is_reported_and_the_handle_recovers():
    mol = synth.tiny_631gs()
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    Dbad = D.clone()
    Dbad[0, 3, 5] = float("nan")
    with pytest.raises(jk.JKError) as e:
        eng.build(Dbad, stats=True)
    assert e.value.code == jk.JK_ERR_NAN
    J, K, _ = eng.build(D, stats=True)
    torch.cuda.synchronize()
    # without stats: the binding's default check synchronises and raises
    with pytest.raises(jk.JKError) as e:
        eng.build(Dbad)
    assert e.value.code == jk.JK_ERR_NAN
    # fully asynchronous: the next call on the handle reports it
    eng.build(Dbad, check=False)
    torch.cuda.synchronize()
    with pytest.raises(jk.JKError) as e:
        eng.build(D)
    assert e.value.code == jk.JK_ERR_NAN
    J, K, _ = eng.build(D)
    eng.close()
    Jr, Kr, _ = oracle.jk(mol)
    assert maxdiff(J.cpu().numpy(), Jr) <= TOL64


def test_autotune_keeps_results_and_writes_its_table(tmp_path, monkeypatch):
    """The autotuner times several fragment shapes per launch; whichever it
    keeps, the build still matches the oracle, and a new handle on the same
    device reads the chosen shapes back from the tuning table."""
    monkeypatch.setenv("JK_TUNING_DIR", str(tmp_path))
    mol = synth.random_small_molecule(7, natm=3, lmax=2, max_nprim=3)
    eng = jk.JK(mol)
    try:
        Dt = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
        rep = eng.autotune(Dt, cutoff=1e-13, max_candidates=3, min_share=0.0)
        assert rep["launches_tuned"] >= 1
        assert rep["candidates_timed"] >= 2 * rep["launches_tuned"]
        assert 0 <= rep["changed"] <= rep["launches_tuned"]
        assert rep["ms_after"] <= rep["ms_before"] + 1e-9
        J, K, _ = eng.build(Dt, cutoff=1e-13, stats=True)
        torch.cuda.synchronize()
    finally:
        eng.close()
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    check(mol, J.cpu().numpy(), Jr, TOL64, "J")
    check(mol, K.cpu().numpy(), Kr, TOL64, "K")
    tables = list(tmp_path.glob("tune_*.txt"))
    assert len(tables) == 1
    lines = tables[0].read_text().split("\n")
    assert len([x for x in lines if x.strip()]) == rep["launches_tuned"]
    # a second handle starts from the stored shapes and still matches
    J2, K2, _ = gpu_jk(mol, cutoff=1e-13)
    check(mol, J2, Jr, TOL64, "J (tuned shapes from the table)")
    check(mol, K2, Kr, TOL64, "K (tuned shapes from the table)")


def _g_molecule(spherical):
    rng = np.random.default_rng(44)
    xyz = np.array([[0.0, 0.0, 0.0], [1.3, -0.2, 0.5]])
    per_atom = [[(0, [3.1, 0.45]), (1, [0.8]), (4, [1.1])],
                [(0, [0.6]), (2, [0.9]), (4, [0.7])]]
    return synth.custom_basis_molecule(xyz, per_atom, rng, spherical=spherical, name="g-pair")


@pytest.mark.parametrize("spherical", [False, True])
def test_g_shells(spherical):
    """g shells (l = 4, up to 9 Rys roots). The (gg|gg), (gg|gd), ... classes
    need more threads per quartet than one CTA holds within the per-thread
    fragment budget, so each quartet is split over several CTAs; the
    Schwarz kernel of the gg pairs is split the same way."""
    mol = _g_molecule(spherical)
    eng = jk.JK(mol)
    Q = jk.jk_schwarz(eng.h)
    eng.close()
    Qr = oracle.schwarz(mol)
    kept = Qr > 1e-18
    assert np.allclose(Q[kept], Qr[kept], rtol=1e-12, atol=0)
    J, K, _ = gpu_jk(mol, cutoff=1e-13)
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    check(mol, J, Jr, TOL64, "J")
    check(mol, K, Kr, TOL64, "K")


def test_g_shells_mixed_precision():
    mol = _g_molecule(False)
    J, K, st = gpu_jk(mol, cutoff=1e-13, precision="mixed")
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    check(mol, J, Jr, TOL_MIXED, "J")
    check(mol, K, Kr, TOL_MIXED, "K")


def test_mixed_precision_at_cutoff_zero_runs_every_quartet_once():
    """With cutoff 0 every tier screens in FP64 (one precision per build), so
    the tiers still partition the quartets exactly."""
    mol = synth.tiny_631gs()
    _, _, s64 = gpu_jk(mol, cutoff=0.0, precision="fp64")
    J, K, sm = gpu_jk(mol, cutoff=0.0, precision="mixed")
    assert sm["quartets_fp64"] + sm["quartets_fp32"] == s64["quartets_fp64"]
    Jr, Kr, _ = oracle.jk(mol, cutoff=0.0)
    check(mol, J, Jr, TOL_MIXED, "J")
    check(mol, K, Kr, TOL_MIXED, "K")
