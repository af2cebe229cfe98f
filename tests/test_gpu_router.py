"""GPU tests of the learned precision router: its forward and backward kernels
against the FP64 CPU reference (oracle/router.py), training, and routed JK
builds judged by the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import router as R
from paper_2507_09772_gb300 import jk, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    jk.load_library()


def random_blob(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    b = jk.JkRouterBlob()
    b.magic = jk.ROUTER_MAGIC
    b.version = 1
    th = (rng.standard_normal(jk.ROUTER_NPARAM) * scale).astype(np.float32)
    for i, v in enumerate(th):
        b.theta[i] = float(v)
    mu = rng.standard_normal(16).astype(np.float32)
    isd = (0.5 + rng.random(16)).astype(np.float32)
    for i in range(16):
        b.mu[i] = float(mu[i])
        b.isd[i] = float(isd[i])
    b.margin = 0.0
    b.quantile = 0.9
    return b, th, mu, isd


def test_forward_matches_cpu_reference():
    b, th, mu, isd = random_blob(1)
    X = np.random.default_rng(2).standard_normal((2000, 12)).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    yd = torch.empty(2000, dtype=torch.float32, device="cuda")
    jk.jk_router_forward(b, Xd, yd)
    ref = R.forward(th, mu, isd, X)
    got = yd.cpu().numpy().astype(np.float64)
    scale = max(1.0, np.abs(ref).max())
    err = np.abs(got - ref) / scale
    # The GPU accumulates in FP32 on the tensor cores, the reference in FP64:
    # an activation within an FP32 rounding of a BF16 tie can round to the
    # other neighbour (one BF16 step, 2^-8 relative) in a few rows.
    assert np.mean(err <= 1e-4) >= 0.99, np.sort(err)[-20:]
    assert err.max() <= 2e-2


@pytest.mark.parametrize("q", [0.5, 0.9])
def test_gradient_matches_cpu_reference(q):
    b, th, mu, isd = random_blob(3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((3000, 12)).astype(np.float32)
    y = rng.standard_normal(3000).astype(np.float32)
    g, loss = jk.jk_router_gradient(b, torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), q)
    lref, gref = R.pinball_grad(th, mu, isd, X, y, q)
    assert loss == pytest.approx(lref, rel=1e-4)
    for lo, hi in [(R.OFF_W1, R.OFF_B1), (R.OFF_B1, R.OFF_W2), (R.OFF_W2, R.OFF_B2), (R.OFF_B2, R.OFF_W3),
                   (R.OFF_W3, R.OFF_B3), (R.OFF_B3, R.NPARAM)]:
        a, r = g[lo:hi].astype(np.float64), gref[lo:hi]
        assert np.linalg.norm(a - r) <= 2e-3 * np.linalg.norm(r) + 1e-9, (lo, hi)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((50000, 12)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - np.abs(X[:, 3]) + 0.05 * rng.standard_normal(50000)).astype(np.float32)
    blob, st = jk.jk_router_train(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"),
                                  steps=600, batch=2048, lr=3e-3, quantile=0.5, seed=7)
    assert st["loss_last"] < 0.4 * st["loss_first"]
    pred = np.zeros(50000, dtype=np.float32)
    pd = torch.empty(50000, dtype=torch.float32, device="cuda")
    jk.jk_router_forward(blob, torch.tensor(X, device="cuda"), pd)
    pred = pd.cpu().numpy()
    assert np.mean(np.abs(pred - y)) < 0.5 * np.mean(np.abs(y - np.median(y)))


def _gpu_build(eng, mol, **kw):
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J, K, st = eng.build(D, stats=True, **kw)
    torch.cuda.synchronize()
    return J.cpu().numpy(), K.cpu().numpy(), st


@pytest.fixture(scope="module")
def trained():
    """Labels from an FP64 build of one molecule, a router trained on them."""
    mol = synth.batched_molecule(6, natm=14)
    eng = jk.JK(mol)
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    cap = 400000
    X = torch.empty((cap, 12), dtype=torch.float32, device="cuda")
    y = torch.empty(cap, dtype=torch.float32, device="cuda")
    n = jk.jk_router_collect(eng.h, [D], 1, 1e-13, [J], [K], X, y)
    n = min(n, cap)
    assert n > 1000
    blob, st = jk.jk_router_train(X[:n], y[:n], steps=800, batch=4096, lr=2e-3, quantile=0.95, seed=11)
    return mol, eng, blob, (J.cpu().numpy(), K.cpu().numpy()), n, st


def test_label_collection_run_is_a_correct_fp64_build(trained):
    mol, eng, blob, (J, K), n, _ = trained
    Jr, Kr, _ = oracle.jk(mol, cutoff=1e-13)
    assert np.abs(J - Jr).max() <= 1e-10 and np.abs(K - Kr).max() <= 1e-10


def test_routed_build_every_quartet_once_and_within_tolerance(trained):
    mol, eng, blob, _, n, st = trained
    assert st["loss_last"] < st["loss_first"]
    J64, K64, s64 = _gpu_build(eng, mol, precision="fp64")
    Jm, Km, sm = _gpu_build(eng, mol, precision="mixed")
    eng.load_router(blob)
    Jr, Kr, sr = _gpu_build(eng, mol, precision="routed")
    # each significant quartet lands in exactly one tier
    assert sr["quartets_fp64"] + sr["quartets_fp32"] == s64["quartets_fp64"]
    assert sm["quartets_fp64"] + sm["quartets_fp32"] == s64["quartets_fp64"]
    # the router moved band quartets to FP32, beyond what Schwarz-only tiering does
    assert sr["quartets_routed"] > 0
    assert sr["quartets_fp32"] == sm["quartets_fp32"] + sr["quartets_routed"]
    Jo, Ko, _ = oracle.jk(mol, cutoff=1e-13)
    assert np.abs(Jr - Jo).max() <= 1e-8
    assert np.abs(Kr - Ko).max() <= 1e-8


def constant_blob(c, margin):
    """A router whose network outputs the constant c for every quartet."""
    b = jk.JkRouterBlob()
    b.magic = jk.ROUTER_MAGIC
    b.version = 1
    for i in range(jk.ROUTER_NPARAM):
        b.theta[i] = 0.0
    b.theta[jk.ROUTER_NPARAM - 1] = float(c)   # b3
    for i in range(16):
        b.mu[i] = 0.0
        b.isd[i] = 1.0
    b.margin = float(margin)
    b.quantile = 0.95
    return b


def test_trained_router_moves_more_than_a_constant_router(trained):
    """What the learned part gains: against the best constant prediction for
    the same pinball quantile (the 0.95 quantile of the training labels) and
    the same margin, the trained router releases more band quartets to FP32,
    and both routed builds stay within 1e-8 of the FP64 oracle."""
    mol, eng, blob, _, n, _ = trained
    cap = 400000
    X = torch.empty((cap, 12), dtype=torch.float32, device="cuda")
    y = torch.empty(cap, dtype=torch.float32, device="cuda")
    D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    m = min(cap, jk.jk_router_collect(eng.h, [D], 1, 1e-13, [J], [K], X, y))
    c = float(np.quantile(y[:m].cpu().numpy(), 0.95))
    Jo, Ko, _ = oracle.jk(mol, cutoff=1e-13)
    eng.load_router(blob)
    Jt, Kt, st_t = _gpu_build(eng, mol, precision="routed")
    eng.load_router(constant_blob(c, blob.margin))
    Jc, Kc, st_c = _gpu_build(eng, mol, precision="routed")
    for Jx, Kx in ((Jt, Kt), (Jc, Kc)):
        assert np.abs(Jx - Jo).max() <= 1e-8 and np.abs(Kx - Ko).max() <= 1e-8
    assert st_t["quartets_routed"] > st_c["quartets_routed"], (st_t["quartets_routed"], st_c["quartets_routed"])
