"""GPU tests of the tensor-core Gram (tcgen05) for BF16, FP16 and E4M3 storage
(and for FP32 storage through its BF16 split, at the end).

The reference is the Gram matrix of the stored codes computed here in FP64:
G = I + (Q diag(s) / Z_scale)^T (Q diag(s) / Z_scale) / mu, with Q the decoded
codes and s the per-column scales the handle reports.  Products of two 16- or
8-bit codes are exact in FP32; the tensor core adds each MMA's products into
the FP32 accumulator with one rounding relative to the running sum, and the
kernel folds the accumulator into double-float after every 128-byte strip (four
MMAs: 64 rows of 16-bit codes, 128 of E4M3).  So an entry carries at most four
FP32 roundings (2^-23 each) of the largest strip partial: <= 4.8e-7 of the
largest entry, reached only when one strip holds everything (small d).
"""
import numpy as np
import pytest

from tests import quantize_ref as QR

pytestmark = pytest.mark.gpu
TOL = 5e-7


def _expected(s, fmt, mu):
    codes, cs = s.stored()
    zs = s.info()["zscale"]
    Zt = QR.decode(codes, fmt) * (cs / zs)[None, :]
    return np.eye(Zt.shape[1]) + Zt.T @ Zt / mu


@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3"])
@pytest.mark.parametrize("d,n", [(37, 5), (1000, 128), (2531, 257), (9000, 300), (20011, 1000)])
def test_tensor_core_gram_matches_fp64(gdwd_lib, fmt, d, n):
    rng = np.random.default_rng(7 * d + n)
    y = np.where(np.arange(n) % 3 == 0, 1.0, -1.0)
    Z = (rng.standard_normal((d, n)) * y).astype(np.float32)
    Z[:, 1] *= 50.0                         # uneven column norms
    mu = 0.7
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store=fmt, mu=mu) as s:
        assert s.info()["gram_tensor_cores"] == 1
        G = s.gram()
        Gref = _expected(s, fmt, mu)
    K, Kref = G - np.eye(n), Gref - np.eye(n)
    err = np.max(np.abs(K - Kref)) / np.max(np.abs(Kref))
    assert err <= TOL, err
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_tensor_core_gram_equals_simt_gram(gdwd_lib, fmt):
    """Both Gram kernels on the same stored data (a slab height that is not a
    multiple of the 128-byte strip, many k-splits)."""
    rng = np.random.default_rng(3)
    d, n = 12345, 700
    y = np.where(np.arange(n) < 300, 1.0, -1.0)
    Z = (rng.standard_t(3, size=(d, n)) * y).astype(np.float32)
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store=fmt, block_rows=72 if fmt == "bf16" else 80) as s:
        assert s.info()["gram_tensor_cores"] == 1
        Gt = s.gram()
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store=fmt, block_rows=72 if fmt == "bf16" else 80, gram_path=1) as s:
        assert s.info()["gram_tensor_cores"] == 0
        Gs = s.gram()
    # the SIMT kernel sums 16-row chunks in FP32 (<= 16 roundings of 2^-24 of the
    # largest partial), so the two may differ by both bounds together
    err = np.max(np.abs(Gt - Gs)) / np.max(np.abs(Gs - np.eye(n)))
    assert err <= TOL + 16 * 2.0 ** -24, err


def test_solve_after_tensor_core_gram(gdwd_lib):
    """A BF16 solve whose factor comes from the tensor-core Gram reaches the same
    solution as one whose factor comes from the SIMT Gram."""
    from paper_2305_12019_gb300 import synth
    inst = synth.gaussian(seed=91, d=8000, n=400, shift=1.0, n_pos=150, q=1.0, C=1.0)
    out = []
    for gp in (0, 1):
        with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="bf16", tol=1e-6, gram_path=gp) as s:
            res, w, _ = s.solve()
            out.append((res[0], w[:, 0]))
    (r0, w0), (r1, w1) = out
    assert r0["status"] == 0 and r1["status"] == 0
    assert abs(r0["primal_obj"] - r1["primal_obj"]) / abs(r1["primal_obj"]) <= 1e-6
    assert np.linalg.norm(w0 - w1) / np.linalg.norm(w1) <= 1e-4


@pytest.mark.parametrize("d,n", [(37, 5), (2531, 257), (20011, 1000)])
def test_fp32_split_gram_matches_fp64(gdwd_lib, d, n):
    """FP32 storage on the tensor cores: each value split into three BF16 terms
    (exact: z = h + m + l up to 2^-24 |z|), six exact products per pair, the h h
    products summed over a 64-row strip in FP32 (four MMAs) and the five smaller
    products (at most 2^-8 of h h) in a second accumulator.  Against the FP64
    Gram of the FP32 data: the accumulator's roundings of each strip's h h
    partial, which need not be round-to-nearest (up to 2^-23 each, of one
    sign), four per strip, plus the dropped terms (below 2^-23 of a product):
    <= 5 * 2^-23 = 6e-7 of the largest entry (1.05e-7 measured at d = 2531
    with one column 50 times the others)."""
    rng = np.random.default_rng(11 * d + n)
    y = np.where(np.arange(n) % 3 == 0, 1.0, -1.0)
    Z = (rng.standard_normal((d, n)) * y).astype(np.float32)
    Z[:, 1] *= 50.0
    mu = 0.7
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store="f32", mu=mu) as s:
        assert s.info()["gram_tensor_cores"] == 1
        G = s.gram()
        zs = s.info()["zscale"]
    Zt = Z.astype(np.float64) / zs
    Kref = Zt.T @ Zt / mu
    err = np.max(np.abs(G - np.eye(n) - Kref)) / np.max(np.abs(Kref))
    assert err <= 6e-7, err
    assert np.array_equal(G, G.T)


def test_fp32_solve_after_split_gram(gdwd_lib):
    """An FP32 solve whose factor comes from the split tensor-core Gram reaches
    the SIMT-Gram solve's solution and iteration count to within the stop rule."""
    from paper_2305_12019_gb300 import synth
    inst = synth.gaussian(seed=92, d=9000, n=600, shift=1.0, n_pos=200, q=1.0, C=2.0)
    out = []
    for gp in (0, 1):
        with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 2.0, store="f32", tol=1e-6, gram_path=gp) as s:
            assert s.info()["gram_tensor_cores"] == (1 if gp == 0 else 0)
            res, w, _ = s.solve()
            out.append((res[0], w[:, 0]))
    (r0, w0), (r1, w1) = out
    assert r0["status"] == 0 and r1["status"] == 0
    assert abs(r0["primal_obj"] - r1["primal_obj"]) / abs(r1["primal_obj"]) <= 1e-6
    assert np.linalg.norm(w0 - w1) / np.linalg.norm(w1) <= 1e-4
