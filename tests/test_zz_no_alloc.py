"""rbo_gram_noalloc: the Gram entry point for callers that cannot let a library
allocate device memory (their HBM belongs to another allocator's pool, or a
cudaMalloc/cudaFree synchronisation is not acceptable where they call it).

It is called here through the C ABI (ctypes) and must agree with rbo_gram, the
allocating entry point, on two calls in a row (the static scratch array keeps
the previous call's contents, so the second call checks that nothing stale is
reused).  This file is collected last so that a failure here does not stop the
rest of the GPU suite; it also passes when run alone in a fresh process, where
the first call performs the per-device set-up."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(rbo, X, Y):
    import torch
    px, n, a, ldx = rbo._mat(X, "X")
    py, n2, b, ldy = rbo._mat(Y, "Y")
    out = torch.full((b, a), float("nan"), dtype=torch.float64, device="cuda")  # column-major a x b
    code = rbo.lib.rbo_gram_noalloc(n, a, px, ldx, b, py, ldy, C.c_void_p(out.data_ptr()),
                                    rbo._stream())
    return code, out.cpu().numpy().T


@pytest.mark.parametrize("n,a,b", [(1_000_003, 60, 5), (20000, 128, 16), (777, 7, 1)])
def test_noalloc_gram_matches_allocating_gram_twice(rbo, n, a, b):
    import torch
    rng = np.random.default_rng(n)
    X = rbo.colmajor(n, a)
    Y = rbo.colmajor(n, b)
    X.copy_(torch.from_numpy(rng.standard_normal((n, a))))
    Y.copy_(torch.from_numpy(rng.standard_normal((n, b))))
    ref = rbo.gram(X, Y)
    scale = float(torch.linalg.vector_norm(X, dim=0).max() * torch.linalg.vector_norm(Y, dim=0).max())
    for _ in range(2):
        code, got = _noalloc(rbo, X, Y)
        assert code == rbo.OK, rbo.lib.rbo_last_error()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-13 * scale


def test_noalloc_rejects_shapes_beyond_its_scratch(rbo):
    import torch
    X = rbo.colmajor(1000, 128)
    Y = rbo.colmajor(1000, 17)     # 128 * 17 > 2048
    X.zero_()
    Y.zero_()
    code, _ = _noalloc(rbo, X, Y)
    assert code == rbo.ERR_ARG
