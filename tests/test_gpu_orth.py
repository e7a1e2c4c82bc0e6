"""GPU parity of the block orthogonalization schemes against the oracle.

Tolerances (float64 path): ||I - Q^T Q||_2 <= 1e-13, ||V - QR||_2/||V||_2 <= 1e-14,
R within 1e-12 (normwise relative) of the oracle when every block has kappa <= 1e4.
For ill-conditioned blocks the computed Q and R depend on rounding at the level
eps * kappa, so parity there is checked through the two error measures, the
per-block conditioning carried by R, and the breakdown reports."""
import numpy as np
import pytest

import synth
from oracle import metrics, orth
from oracle.sketch import Sketch as OSketch

pytestmark = pytest.mark.gpu


def run(rbo, scheme, V, s, s_hat=None, v0=False, precision=0, d=None):
    from gpu_util import to_dev, to_host
    n, c = V.shape
    d = d or 4 * (c + 1 - (1 if v0 else 0) + (1 if v0 else 0))
    sk = rbo.sketch_create(n, d, 8, 42)
    Vd = to_dev(V)
    if scheme == "one":
        out = rbo.block_orth_one_stage(sk, Vd, s, v0=v0, precision=precision, raise_on_error=False)
    elif scheme == "two":
        out = rbo.block_orth_two_stage(sk, Vd, s, s_hat, v0=v0, precision=precision,
                                       raise_on_error=False)
    else:
        out = rbo.block_orth_cholqr2(Vd, s, v0=v0, raise_on_error=False)
    return to_host(Vd), out


def oracle(scheme, V, s, s_hat=None, v0=False, d=None):
    """The C++ oracle's result for the same input and sketch (Q, R, ok, breakdown)."""
    from oracle import cpp_oracle as cpp
    n, c = V.shape
    d = d or 4 * (c + 1 - (1 if v0 else 0) + (1 if v0 else 0))
    if scheme == "one":
        return cpp.block_orth_one_stage(V, s, d=d, v0=v0)
    if scheme == "two":
        return cpp.block_orth_two_stage(V, s, s_hat, d=d, v0=v0)
    return cpp.block_orth_one_stage(V, s, intra="cholqr2", v0=v0)


@pytest.mark.parametrize("scheme,s_hat", [("one", None), ("two", 30), ("two", 10), ("cholqr2", None)])
@pytest.mark.parametrize("n", [20000, 12347, 1001])
def test_well_conditioned_elementwise(rbo, scheme, s_hat, n):
    V = synth.glued_blocks(n, 12, 5, 1e4, seed=n, v0=True)
    Q, out = run(rbo, scheme, V, 5, s_hat, v0=True)
    ref = oracle(scheme, V, 5, s_hat, v0=True)
    assert out.info["status"] == 0 and ref.ok
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12
    assert np.abs(Q - ref.Q).max() <= 1e-9
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    assert np.allclose(np.tril(out.R, -1), 0.0) and (np.diag(out.R) > 0).all()


@pytest.mark.parametrize("scheme,s_hat", [("one", None), ("two", 30), ("two", 60)])
def test_config0_kappa_1e10(rbo, scheme, s_hat):
    # 20000 x 60, 12 blocks of 5 with kappa = 1e10 each, sparse-sign d = 4*61, zeta 8, seed 42
    V = synth.glued_blocks(20000, 12, 5, 1e10, seed=0)
    Q, out = run(rbo, scheme, V, 5, s_hat, d=244)
    assert out.info["status"] == 0
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    ref = oracle(scheme, V, 5, s_hat, d=244)
    for j in range(12):
        c_gpu = metrics.cond2(out.R[5 * j:5 * j + 5, 5 * j:5 * j + 5])
        c_ref = metrics.cond2(ref.R[5 * j:5 * j + 5, 5 * j:5 * j + 5])
        assert abs(np.log10(c_gpu) - np.log10(c_ref)) < 0.01
    # R is unique: agreement is limited by conditioning (eps * kappa)
    assert metrics.rel_diff(out.R, ref.R) <= 1e-4


def test_cholqr2_breakdown_reported(rbo):
    V = synth.glued_blocks(20000, 12, 5, 1e10, seed=0)
    Q, out = run(rbo, "cholqr2", V, 5)
    ref = oracle("cholqr2", V, 5)
    assert not ref.ok
    assert out.info["status"] in (rbo.ERR_CHOL_BREAKDOWN, rbo.ERR_LOST_ORTHOGONALITY)
    # every block has kappa = 1e10 (kappa^2 eps >> 1): the deciding pivots are at
    # rounding level, so which block fails first depends on the summation order (the
    # oracle fails at block 0); a breakdown must be reported at one of the 12 blocks
    assert 0 <= out.info["breakdown_block"] < 12
    assert out.info["breakdown_stage_name"] in ("intra", "intra2", "final")
    if out.info["status"] == rbo.ERR_CHOL_BREAKDOWN:
        assert 0 <= out.info["breakdown_column"] < 5


@pytest.mark.parametrize("kappa", [1e4, 1e8, 1e12, 1e14])
def test_two_stage_kappa_sweep(rbo, kappa):
    V = synth.glued_blocks(30000, 12, 5, kappa, seed=17, v0=True)
    Q, out = run(rbo, "two", V, 5, 30, v0=True)
    assert out.info["status"] == 0
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14


@pytest.mark.parametrize("scheme", ["one", "two"])
def test_mixed_precision_meets_fp64_bounds_at_moderate_kappa(rbo, scheme):
    V = synth.glued_blocks(20000, 12, 5, 1e4, seed=9, v0=True)
    Q, out = run(rbo, scheme, V, 5, 30, v0=True, precision=rbo.PREC_MIXED)
    ref = oracle(scheme, V, 5, 30, v0=True)
    assert out.info["status"] == 0
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12


@pytest.mark.parametrize("n,s,nb", [(7, 1, 5), (64, 5, 2), (65, 5, 2), (129, 16, 8), (3, 3, 1)])
def test_edge_shapes(rbo, n, s, nb):
    V = synth.glued_blocks(n, nb, s, 10.0, seed=n)
    Q, out = run(rbo, "one", V, s, d=max(4 * (nb * s + 1), 16))
    ref = oracle("one", V, s, d=max(4 * (nb * s + 1), 16))
    assert out.info["status"] == 0
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12
    assert metrics.orth_error(Q) <= 1e-13


def test_invalid_arguments_are_rejected(rbo):
    import torch
    from gpu_util import to_dev
    V = to_dev(np.random.default_rng(0).standard_normal((100, 12)))
    sk = rbo.sketch_create(100, 52, 8, 42)
    with pytest.raises(rbo.RboError) as e:
        rbo.block_orth_one_stage(sk, V, 5)  # 12 not a multiple of 5
    assert e.value.code == rbo.ERR_ARG
    with pytest.raises(rbo.RboError):
        rbo.block_orth_two_stage(sk, V, 4, 6)  # s does not divide s_hat
    small = rbo.sketch_create(10, 52, 8, 42)
    with pytest.raises(rbo.RboError):
        rbo.block_orth_one_stage(small, V, 4)  # sketch too short for n


def test_rank_deficient_block_reports_breakdown(rbo):
    V = synth.glued_blocks(5000, 3, 5, 1e4, seed=1)
    V[:, 7] = V[:, 6]  # exact duplicate column inside block 1
    Q, out = run(rbo, "one", V, 5, d=64)
    assert out.info["status"] == rbo.ERR_CHOL_BREAKDOWN
    assert out.info["breakdown_block"] == 1


def test_nan_input_reports_breakdown_not_silence(rbo):
    V = synth.glued_blocks(5000, 2, 5, 1e2, seed=2)
    V[10, 3] = np.nan
    Q, out = run(rbo, "one", V, 5, d=64)
    assert out.info["status"] == rbo.ERR_CHOL_BREAKDOWN


@pytest.mark.parametrize("scheme", ["one", "two"])
@pytest.mark.parametrize("kappa", [1e12, 1e14])
def test_mixed_precision_redoes_failed_blocks_in_float64(rbo, scheme, kappa):
    # float32 sketching cannot precondition blocks with kappa >> 1/eps_32: such a block
    # (two-stage: big panel) is redone in float64 from a copy of its input, float64
    # stays on, and the call ends in status 0 at the float64 tolerances
    V = synth.glued_blocks(20000, 12, 5, kappa, seed=13, v0=True)
    Q, out = run(rbo, scheme, V, 5, 30, v0=True, precision=rbo.PREC_MIXED)
    assert out.info["status"] == 0, out.info
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    Q64, out64 = run(rbo, scheme, V, 5, 30, v0=True)
    assert out64.info["fallbacks"] == 0
    if kappa >= 1e14:
        assert out.info["fallbacks"] >= 1


@pytest.mark.parametrize("scheme,s_hat", [("one", None), ("two", 30), ("two", 60)])
@pytest.mark.parametrize("kappa", [1e4, 1e10, 1e14])
def test_df64_meets_the_fp64_tolerances(rbo, scheme, s_hat, kappa):
    # float32-pair arithmetic (about 48 significant bits per operation) must give the
    # float64-path results: orthogonality 1e-13, backward error 1e-14, and R within
    # 1e-12 of the oracle for kappa <= 1e4
    if s_hat == 60:
        V = synth.glued_blocks(20000, 12, 5, kappa, seed=31)
    else:
        V = synth.glued_blocks(20000, 12, 5, kappa, seed=31, v0=True)
    v0 = s_hat != 60
    Q, out = run(rbo, scheme, V, 5, s_hat, v0=v0, precision=rbo.PREC_DF64)
    assert out.info["status"] == 0
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    if kappa <= 1e4:
        ref = oracle(scheme, V, 5, s_hat, v0=v0)
        assert metrics.rel_diff(out.R, ref.R) <= 1e-12


@pytest.mark.parametrize("n", [1001, 12347])
def test_df64_ragged_sizes(rbo, n):
    V = synth.glued_blocks(n, 12, 5, 1e8, seed=n, v0=True)
    for scheme in ("one", "two"):
        Q, out = run(rbo, scheme, V, 5, 30, v0=True, precision=rbo.PREC_DF64)
        assert out.info["status"] == 0
        assert metrics.orth_error(Q) <= 1e-13
        assert metrics.backward_error(V, Q, out.R) <= 1e-14


# --- two-stage with BCGS-PIP preprocessing (Section 7.1) ---------------------------
@pytest.mark.parametrize("n,s_hat", [(20000, 30), (12347, 10)])
def test_two_stage_pip_matches_oracle(rbo, n, s_hat):
    from gpu_util import to_dev, to_host
    V = synth.glued_blocks(n, 12, 5, 1e4, seed=n + 3, v0=True)
    Vd = to_dev(V)
    out = rbo.block_orth_two_stage(None, Vd, 5, s_hat, v0=True, preproc=rbo.PREPROC_PIP)
    Q = to_host(Vd)
    from oracle import cpp_oracle as cpp
    ref = cpp.block_orth_two_stage(V, 5, s_hat, v0=True, preproc="pip")
    assert out.info["status"] == 0 and ref.ok
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12
    assert np.abs(Q - ref.Q).max() <= 1e-9
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14


def test_two_stage_pip_breakdown_reported(rbo):
    # kappa^2 eps >> 1: the Pythagorean Gram loses positive definiteness; both the
    # oracle and the GPU report a breakdown in the preprocessing (RandBCGS2 does not)
    from gpu_util import to_dev
    V = synth.glued_blocks(20000, 12, 5, 1e10, seed=2)
    out = rbo.block_orth_two_stage(None, to_dev(V), 5, 30, preproc=rbo.PREPROC_PIP,
                                   raise_on_error=False)
    ref = orth.block_orth_two_stage(V, 5, 30, None, preproc="pip")
    assert not ref.ok and ref.breakdown_where == "bcgs-pip"
    assert out.info["status"] == rbo.ERR_CHOL_BREAKDOWN
    assert out.info["breakdown_stage_name"] == "preproc"
    assert 0 <= out.info["breakdown_block"] < 2


# --- Gaussian and Count-Gauss sketches in the randomized schemes (Section 5.2) ------
@pytest.mark.parametrize("kind", ["gauss", "count_gauss"])
def test_gaussian_sketch_schemes_match_oracle(rbo, kind):
    from gpu_util import to_dev, to_host
    from oracle.sketch import CountGaussSketch, GaussianSketch
    n = 20000

    def make(d):
        if kind == "gauss":
            return (rbo.sketch_create(n, d, seed=42, kind=rbo.SKETCH_GAUSSIAN),
                    GaussianSketch(n, d, 42))
        di = 4 * d * d // 10
        return (rbo.sketch_create(n, d, seed=42, kind=rbo.SKETCH_COUNT_GAUSS, d_inner=di),
                CountGaussSketch(n, d, di, 42))

    # kappa = 1e4: R is unique, so the GPU and the oracle agree to rounding
    V = synth.glued_blocks(n, 12, 5, 1e4, seed=1)
    sk, osk = make(10)
    Vd = to_dev(V)
    out = rbo.block_orth_one_stage(sk, Vd, 5)
    ref = orth.block_orth_one_stage(V, 5, osk)
    assert out.info["status"] == 0 and ref.ok
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12
    # kappa = 1e10 (CholQR2 fails): O(eps) with either map, one- and two-stage
    V = synth.glued_blocks(n, 12, 5, 1e10, seed=0)
    for scheme, d in (("one", 10), ("two", 60)):
        sk, _ = make(d)
        Vd = to_dev(V)
        if scheme == "one":
            out = rbo.block_orth_one_stage(sk, Vd, 5)
        else:
            out = rbo.block_orth_two_stage(sk, Vd, 5, 30)
        Q = to_host(Vd)
        assert out.info["status"] == 0
        assert metrics.orth_error(Q) <= 1e-13
        assert metrics.backward_error(V, Q, out.R) <= 1e-14
