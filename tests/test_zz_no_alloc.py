"""The Gram entry point that allocates nothing (gdwd_gram_noalloc).

It is for callers that cannot allocate device memory when they need the
product, so its scratch is a fixed array inside the library that every call
reuses.  The test calls it twice in a row through the C-ABI, on data of two
different shapes, and checks each result against the Gram matrix built by the
ordinary (allocating) path with its SIMT kernel, gdwd_create (gram_path = 1) +
gdwd_gram, and against the FP64 product, within the tolerance of the SIMT Gram
tests; it must pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference_gram(gdwd_lib, Z):
    """Z^T Z from the allocating path's SIMT Gram: gdwd_gram returns I + Z~^T Z~ with Z~ = Z / Z_scale."""
    n = Z.shape[1]
    y = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store="f32", mu=1.0, gram_path=1) as s:
        G = s.gram()
        zs = s.info()["zscale"]
    return (G - np.eye(n)) * zs * zs


def test_gram_noalloc_matches_allocating_path(gdwd_lib):
    import torch
    rng = np.random.default_rng(2024)
    for d, n in [(3001, 257), (1000, 1500)]:     # two calls in a row share the scratch array
        Zh = rng.standard_normal((d, n)).astype(np.float32)
        Zd = torch.from_numpy(np.ascontiguousarray(Zh.T)).cuda()      # n x d: rows are the columns of Z
        Zcm = torch.as_strided(Zd, (d, n), (1, d))
        K = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        gdwd_lib.gram_noalloc(Zcm, K)
        torch.cuda.synchronize()
        got = K.cpu().numpy()
        ref = _reference_gram(gdwd_lib, Zh)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert np.all(np.isfinite(got))
        assert err <= 5e-8, (d, n, err)
        assert np.array_equal(got, got.T)
        # and directly against the FP64 product of the same FP32 data, so that an
        # error both paths share cannot hide
        exact = Zh.astype(np.float64).T @ Zh.astype(np.float64)
        err64 = np.abs(got - exact).max() / np.abs(exact).max()
        assert err64 <= 5e-8, (d, n, err64)


def test_gram_noalloc_rejects_oversize(gdwd_lib):
    """n beyond the fixed scratch (n > 2048) is refused by the library before any GPU work."""
    import ctypes
    import torch
    big = torch.as_strided(torch.zeros(8 * 2049, dtype=torch.float32, device="cuda"), (8, 2049), (1, 8))
    K = torch.zeros(2049 * 2049, dtype=torch.float64, device="cuda")
    with pytest.raises(gdwd_lib.GdwdError):
        gdwd_lib.gram_noalloc(big, K)
    # the C entry point itself, with n so large that n * n would overflow int64
    lib = gdwd_lib.load()
    st = lib.gdwd_gram_noalloc(ctypes.c_void_p(big.data_ptr()), 8, 1 << 40, 8, ctypes.c_void_p(K.data_ptr()), None)
    assert st == 1   # GDWD_EINVAL


def test_gram_noalloc_rejects_small_output(gdwd_lib):
    """An output K with fewer than n * n elements is refused before anything is launched."""
    import torch
    Z = torch.as_strided(torch.ones(64 * 100, dtype=torch.float32, device="cuda"), (64, 100), (1, 64))
    K = torch.zeros(100 * 100 - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        gdwd_lib.gram_noalloc(Z, K)
    Kf = torch.zeros(100 * 100, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        gdwd_lib.gram_noalloc(Z, Kf)
