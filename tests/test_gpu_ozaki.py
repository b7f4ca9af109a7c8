"""The emulated FP64 rank-k update (gj_gemm_update_emulated: BF16 tcgen05 tensor cores,
exact digit splitting) against an FP64 product computed on the host.

Error bound (derived from the splitting): every entry of L is rounded to 8S - 1 fractional
bits of its row scale 2^(e_i + 1) and written as S balanced base-256 digits in [-128, 128]
(error <= 2^(e_i - 8S)), every entry of U likewise with its column scale (together
<= 2 K 2^(e_i + f_j - 8S) over the k sum, to first order); the digit pairs with s + t >= S
are dropped (at most S - 1 pairs per group, digit products <= 2^14, weights
2^-8(s+t+2) of 2^(e_i + f_j + 2): < 1.01 (S - 1) K 2^(e_i + f_j - 8S)); the kept products are
summed exactly, and the integer combination drops the bits of the two lowest groups below
2^(e_i + f_j - 55) (< 2 2^(e_i + f_j - 55)).  The entry (i, j) of L U is therefore off by
less than (S + 2) K 2^(e_i + f_j - 8S) + 2^(e_i + f_j - 54), plus the FP64 roundings of the
int64 -> FP64 conversion and the final add (<= 4 K eps sum_k |L_ik||U_kj| + 2 eps |C_new|).
The test checks exactly that bound.
"""
import numpy as np
import pytest

import paper_1401_7962_gb300 as gj

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EPS = float(np.finfo(np.float64).eps)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_7962_gb300 import _build
    _build.build()
    gj.lib()


def scale_exp(x, axis):
    """e with max |x| < 2^e along `axis` (row / column scales of the splitting)."""
    m = np.max(np.abs(x), axis=axis)
    e = np.floor(np.log2(np.where(m > 0, m, 1.0))).astype(np.int64) + 1
    return np.where(m > 0, e, -100000)


def run(M, N, K, S, rng, ldl_pad=0, scale_rows=False):
    L = rng.standard_normal((M, K))
    if scale_rows:
        L *= np.exp2(rng.integers(-30, 30, size=(M, 1)))
    U = rng.standard_normal((K, N))
    C = rng.standard_normal((M, N))
    Lb = np.zeros((M + ldl_pad, K), order="F")
    Lb[:M] = L
    dL = torch.from_numpy(Lb).cuda()
    dU = torch.from_numpy(np.asfortranarray(U)).cuda()
    dC = torch.from_numpy(np.asfortranarray(C)).cuda()
    L_ = gj.lib()
    st = L_.gj_gemm_update_emulated(M, N, K, dL.data_ptr(), M + ldl_pad, dU.data_ptr(), K, dC.data_ptr(), M, S, None)
    assert st == 0, (st, gj.last_error())
    got = dC.cpu().numpy()
    ref = C + L @ U
    e = scale_exp(L, 1)[:, None]
    f = scale_exp(U, 0)[None, :]
    bound = (S + 2.0) * K * np.exp2((e + f - 8 * S).astype(np.float64)) + np.exp2((e + f - 54).astype(np.float64)) + \
        2 * EPS * np.abs(ref) + 4 * K * EPS * (np.abs(L) @ np.abs(U))
    return got, ref, bound


@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (128, 64, 16), (300, 200, 100), (257, 129, 64), (5, 3, 1),
                                   (1000, 1000, 128), (129, 65, 127)])
@pytest.mark.parametrize("S", [7, 8])
def test_emulated_update_within_bound(M, N, K, S):
    rng = np.random.default_rng(M * 7 + N * 3 + K + S)
    got, ref, bound = run(M, N, K, S, rng)
    err = np.abs(got - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("M,N,K,S", [(256, 40000, 32, 1), (256, 40000, 32, 8), (130, 30000, 128, 8),
                                     (1100, 3000, 128, 8), (2048, 2048, 64, 3)])
def test_emulated_update_many_tiles_per_cta(M, N, K, S):
    """Grids of several tiles per CTA: tile columns change inside a CTA's range (the U slices
    are reloaded), and with K <= 64 and S = 1 the producer runs tiles ahead of the MMAs."""
    rng = np.random.default_rng(M + N + K + S)
    got, ref, bound = run(M, N, K, S, rng)
    err = np.abs(got - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_emulated_update_scaled_rows_and_lda():
    rng = np.random.default_rng(11)
    got, ref, bound = run(384, 192, 128, 8, rng, ldl_pad=9, scale_rows=True)
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5])
def test_fewer_slices_obey_their_bound(S):
    rng = np.random.default_rng(20 + S)
    got, ref, bound = run(256, 128, 128, S, rng)
    assert np.all(np.abs(got - ref) <= bound)


def test_emulated_update_argument_errors():
    L_ = gj.lib()
    assert L_.gj_gemm_update_emulated(4, 4, 129, 1, 4, 1, 129, 1, 4, 8, None) == gj.ERR_ARG
    assert L_.gj_gemm_update_emulated(4, 4, 4, 1, 4, 1, 4, 1, 4, 9, None) == gj.ERR_ARG
    assert L_.gj_gemm_update_emulated(4, 4, 4, 1, 3, 1, 4, 1, 4, 8, None) == gj.ERR_ARG
    assert L_.gj_gemm_update_emulated(0, 4, 4, 0, 1, 0, 4, 0, 1, 8, None) == gj.OK


def test_peak_probes_report_plausible_rates():
    """gj_measure_peaks (the benchmark's FP64 roofline denominators): finite, positive rates;
    the FP32 FMA rate well above the FP64 rates on this part."""
    p = gj.measure_peaks()
    assert p["sm_count"] > 0 and p["max_clock_mhz"] > 0
    for k in ("fp64_fma_gflops", "fp64_mma_gflops", "fp32_fma_gflops"):
        assert np.isfinite(p[k]) and p[k] > 10.0, (k, p[k])
    assert p["fp32_fma_gflops"] > 4 * p["fp64_fma_gflops"]
