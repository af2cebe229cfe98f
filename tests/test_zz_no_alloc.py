"""The allocation-free gradient entry point (jk_router_gradient_noalloc).

Callers that must not call cudaMalloc (applications whose own allocator
owns all device memory, or loops that cannot afford the device-wide
synchronisation of cudaFree) use this variant; its scratch is a fixed array
inside the library. It must give
the same loss and gradient as jk_router_gradient, call after call, even
though every call reuses the same scratch. This file is collected last so a
stop-at-first-failure run has executed every other test before it.
"""
import numpy as np
import pytest

from paper_2507_09772_gb300 import jk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_blob(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    b = jk.JkRouterBlob()
    b.magic = jk.ROUTER_MAGIC
    b.version = 1
    th = (rng.standard_normal(jk.ROUTER_NPARAM) * scale).astype(np.float32)
    ctypes_arr = b.theta
    for i, v in enumerate(th):
        ctypes_arr[i] = float(v)
    for i in range(16):
        b.mu[i] = float(rng.standard_normal())
        b.isd[i] = float(0.5 + rng.random())
    return b


def rel_err(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b.astype(np.float64)) / max(np.linalg.norm(b), 1e-30))


def test_noalloc_gradient_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    jk.load_library()
    rng = np.random.default_rng(17)
    cases = []
    for seed, n, q in ((1, 5000, 0.9), (2, 1234, 0.5)):   # second call: other weights, fewer rows
        X = torch.tensor(rng.standard_normal((n, 12)).astype(np.float32), device="cuda")
        y = torch.tensor(rng.standard_normal(n).astype(np.float32), device="cuda")
        cases.append((make_blob(seed), X, y, q))
    for blob, X, y, q in cases:
        g_ref, l_ref = jk.jk_router_gradient(blob, X, y, q)
        g, l = jk.jk_router_gradient_noalloc(blob, X, y, q)
        assert l == pytest.approx(l_ref, rel=1e-4)
        assert rel_err(g, g_ref) <= 2e-3
        assert np.isfinite(g).all()


def test_noalloc_rejects_more_rows_than_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    n = 65537
    X = torch.zeros((n, 12), dtype=torch.float32, device="cuda")
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(jk.JKError) as e:
        jk.jk_router_gradient_noalloc(make_blob(3), X, y, 0.9)
    assert e.value.code == jk.JK_ERR_UNSUPPORTED
    assert "65536" in str(e.value)
