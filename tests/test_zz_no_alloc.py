"""rbo_gram_noalloc: the Gram entry point for callers that cannot let a library
allocate device memory (their HBM belongs to another allocator's pool, or a
cudaMalloc/cudaFree synchronisation is not acceptable where they call it).

It is called here through the C ABI (ctypes) and must agree with rbo_gram, the
allocating entry point, on two calls in a row.  The static scratch array keeps the
previous call's contents, so the second call uses other data and another shape (a
different grid and reduction-group count) and each result is checked against
rbo_gram on that call's own inputs.  A further test checks the property the entry
point exists for: with the library's workspace released, a call leaves the device's
free memory unchanged.  This file is collected last so that a failure here does not
stop the rest of the GPU suite; it also passes when run alone in a fresh process,
where the first call performs the per-device set-up."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(rbo, X, Y, out=None):
    import torch
    px, n, a, ldx = rbo._mat(X, "X")
    py, n2, b, ldy = rbo._mat(Y, "Y")
    if out is None:
        out = torch.full((b, a), float("nan"), dtype=torch.float64, device="cuda")  # column-major a x b
    else:
        out.fill_(float("nan"))
    code = rbo.lib.rbo_gram_noalloc(n, a, px, ldx, b, py, ldy, C.c_void_p(out.data_ptr()),
                                    rbo._stream())
    return code, out.cpu().numpy().T


def _inputs(rbo, n, a, b, seed):
    import torch
    rng = np.random.default_rng(seed)
    X = rbo.colmajor(n, a)
    Y = rbo.colmajor(n, b)
    X.copy_(torch.from_numpy(rng.standard_normal((n, a))))
    Y.copy_(torch.from_numpy(rng.standard_normal((n, b))))
    scale = float(torch.linalg.vector_norm(X, dim=0).max() * torch.linalg.vector_norm(Y, dim=0).max())
    return X, Y, scale


@pytest.mark.parametrize("first,second", [((1_000_003, 60, 5), (777, 7, 1)),
                                          ((777, 7, 1), (20000, 128, 16)),
                                          ((20000, 128, 16), (1_000_003, 60, 5))])
def test_noalloc_gram_matches_allocating_gram_on_two_calls(rbo, first, second):
    for k, (n, a, b) in enumerate((first, second)):
        X, Y, scale = _inputs(rbo, n, a, b, seed=1000 * k + n)
        ref = rbo.gram(X, Y)
        code, got = _noalloc(rbo, X, Y)
        assert code == rbo.OK, rbo.lib.rbo_last_error()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-13 * scale, (n, a, b)


def test_noalloc_gram_allocates_nothing(rbo):
    import torch
    X, Y, scale = _inputs(rbo, 300_001, 40, 8, seed=7)
    ref = rbo.gram(X, Y)
    out = torch.empty((8, 40), dtype=torch.float64, device="cuda")
    code, _ = _noalloc(rbo, X, Y, out)          # per-device set-up happens at the latest here
    assert code == rbo.OK
    assert rbo.release_workspace() == rbo.OK      # no library arena from here on
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    code = rbo.lib.rbo_gram_noalloc(300_001, 40, C.c_void_p(X.data_ptr()), X.stride(1), 8,
                                    C.c_void_p(Y.data_ptr()), Y.stride(1), C.c_void_p(out.data_ptr()),
                                    rbo._stream())
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert code == rbo.OK, rbo.lib.rbo_last_error()
    assert free1 == free0, (free0, free1)
    got = out.cpu().numpy().T
    assert np.abs(got - ref).max() <= 1e-13 * scale


def test_noalloc_rejects_shapes_beyond_its_scratch(rbo):
    X = rbo.colmajor(1000, 128)
    Y = rbo.colmajor(1000, 17)     # 128 * 17 > 2048
    X.zero_()
    Y.zero_()
    code, _ = _noalloc(rbo, X, Y)
    assert code == rbo.ERR_ARG
