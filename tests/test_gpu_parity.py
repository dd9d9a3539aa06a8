"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerance (forward and inverse, FP64 form): max |c_gpu - c_oracle| <= 1e-12 * ||c_in||_1,
the bound stated for this library.  At full size (N = 2^16, 2^18) the oracle
evaluates sampled grid values in double-double; the GPU result is checked
through the identities that hold at any size:
  forward:  sum_k c_cheb_k T_k(x_j) = sum_n c_jac_n P_n(x_j) at sampled x_j
  inverse:  sum_n c_jac_n P_n(x_j)  = sum_k c_cheb_k T_k(x_j) at sampled x_j
and by the round trip inverse(forward(c)) = c.
"""
import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12

PARAMS = [(0.1, -0.3), (0.45, 0.45), (-0.45, 0.2), (0.0, 0.0), (0.125, 0.375), (-0.5, -0.5), (0.5, 0.5),
          (0.5, -0.5), (-0.5, 0.3), (0.37, -0.5)]


@pytest.fixture(scope="module")
def cjt():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt as mod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def l1(c):
    return float(np.abs(c).sum())


def run_fwd(cjt, plan, c):
    y = cjt.cjt_forward(plan, dev(c))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def run_inv(cjt, plan, c):
    y = cjt.cjt_inverse(plan, dev(c))
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("alpha,beta", PARAMS)
@pytest.mark.parametrize("N", [1, 2, 4, 8, 64, 256, 1024, 4096])
def test_forward_matches_oracle(cjt, orc, N, alpha, beta):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + N)
    plan = cjt.Plan(N, alpha, beta)
    got = run_fwd(cjt, plan, c)
    ref = orc.forward(c, alpha, beta)
    assert np.max(np.abs(got - ref)) <= TOL * l1(c)


@pytest.mark.parametrize("alpha,beta", PARAMS)
@pytest.mark.parametrize("N", [1, 2, 4, 8, 64, 256, 1024, 4096])
def test_inverse_matches_oracle(cjt, orc, N, alpha, beta):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 7 * N)
    plan = cjt.Plan(N, alpha, beta)
    got = run_inv(cjt, plan, c)
    ref = orc.inverse(c, alpha, beta)
    assert np.max(np.abs(got - ref)) <= TOL * l1(c)


@pytest.mark.parametrize("opts", [dict(M=3), dict(M=5), dict(M=10), dict(M=13), dict(M=20), dict(use_asy=-1),
                                  dict(seg_len=32), dict(seg_len=96), dict(ratio=0.5), dict(ratio=0.2),
                                  dict(M=13, seg_len=64), dict(rec_store=1), dict(rec_store=1, seg_len=64, M=5),
                                  dict(rec_store=1, use_asy=-1)])
def test_options_do_not_change_the_result(cjt, orc, opts):
    """The partition, M and the work split change only the rounding (Sec. 2.2)."""
    N, a, b = 4096, 0.1, -0.3
    c = inputs.decaying_coefficients(N, 1.5, 99)
    plan = cjt.Plan(N, a, b, **opts)
    info = plan.info()
    assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, a, b))) <= TOL * l1(c), info
    assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, a, b))) <= TOL * l1(c), info


@pytest.mark.parametrize("opts", [dict(seg_whole=1024), dict(seg_whole=8192, M=13),
                                  dict(seg_whole=1 << 22, rec_store=1), dict(seg_whole=2048, precision=2),
                                  dict(seg_whole=2048, precision=2, rec_store=1), dict(seg_whole=700, fold_check=1)])
@pytest.mark.parametrize("N", [4096, 6000])
def test_whole_rows_match_oracle(cjt, orc, N, opts):
    """seg_whole: rows whose recurrence spans at most that many degrees run as one work item
    (no segment states); the transposed items of such rows span several of the reduction's
    degree segments.  The result stays within the tolerance of the oracle (alpha = beta adds
    the parity fold with stored values)."""
    opts = dict(opts, seg_len=256)
    a, b = (0.2, 0.2) if opts.pop("fold_check", 0) else (0.1, -0.3)
    if a == b:
        opts["rec_store"] = 1
    c = inputs.decaying_coefficients(N, 1.5, 4100 + N)
    plan = cjt.Plan(N, a, b, **opts)
    assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, a, b))) <= TOL * l1(c), opts
    assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, a, b))) <= TOL * l1(c), opts


def test_partition_matches_paper_shape(cjt):
    """N = 1024, (0.1, -0.3), M = 7: two asymptotic blocks and most of the matrix by ASY."""
    plan = cjt.Plan(1024, 0.1, -0.3, M=7)
    info = plan.info()
    assert info["n_M"] > 50 and info["nblk_fwd"] >= 1
    assert info["rec_steps_fwd"] < 0.6 * 1025 ** 2


@pytest.mark.parametrize("N", [1 << 14])
def test_forward_inverse_16384_elementwise(cjt, orc, N):
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 1001)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + 1)
    plan = cjt.Plan(N, a, b)
    assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, a, b))) <= TOL * l1(c)
    assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, a, b))) <= TOL * l1(c)


def test_forward_inverse_65536_elementwise(cjt, orc):
    N = 1 << 16
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 1002)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + 2)
    plan = cjt.Plan(N, a, b)
    assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, a, b))) <= TOL * l1(c)
    assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, a, b))) <= TOL * l1(c)


@pytest.mark.parametrize("logN", [16, 18])
def test_full_size_properties(cjt, orc, logN):
    """At any size: value-space identities at sampled Lobatto points (double-double oracle),
    the exact first inverse coefficient c_jac_0 = sum_k c_k mu_k / mu_0 (Eq. cjintdefn, n = 0),
    and the round trip inverse(forward(c)) = c."""
    N = 1 << logN
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 1000 + logN)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + logN)
    plan = cjt.Plan(N, a, b)
    rng = inputs.rng(5)
    j = np.unique(np.concatenate([np.arange(0, 40), N - np.arange(0, 40), rng.integers(0, N + 1, 400)]))
    # forward: sum_k c_cheb_k T_k(x_j) = sum_n c_n P_n(x_j)
    fwd = run_fwd(cjt, plan, c)
    y_ref = orc.jacobi_series(c, a, b, j, N)
    y_got = orc.cheb_series(fwd, j, N)
    assert np.max(np.abs(y_got - y_ref)) <= TOL * l1(c)
    # inverse: sum_n c_jac_n P_n(x_j) = sum_k c_k T_k(x_j).  A coefficient error within the
    # tolerance moves the value at x_j by at most TOL ||c||_1 sum_n |P_n(x_j)|.
    inv = run_inv(cjt, plan, c)
    v_ref = orc.cheb_series(c, j, N)
    v_got = orc.jacobi_series(inv, a, b, j, N)
    for q in range(0, j.size, 37):
        bound = TOL * l1(c) * np.abs(orc.jacobi_values(N, a, b, int(j[q]), N)).sum()
        assert abs(v_got[q] - v_ref[q]) <= bound
    mu = orc.moments(N, a, b)
    assert abs(inv[0] - np.dot(c, mu) / mu[0]) <= TOL * l1(c)
    # round trips
    back = run_inv(cjt, plan, fwd)
    assert np.max(np.abs(back - c)) <= TOL * l1(c)
    again = run_fwd(cjt, plan, inv)
    assert np.max(np.abs(again - c)) <= TOL * l1(c)


def test_in_place_and_determinism(cjt, orc):
    N, a, b = 2048, 0.3, -0.2
    c = inputs.decaying_coefficients(N, 1.0, 3)
    plan = cjt.Plan(N, a, b)
    x = dev(c)
    y1 = cjt.cjt_forward(plan, x).cpu().numpy()
    y2 = cjt.cjt_forward(plan, x).cpu().numpy()
    assert np.array_equal(y1, y2)
    z = dev(c)
    cjt.cjt_forward(plan, z, z)   # aliasing input and output
    torch.cuda.synchronize()
    assert np.array_equal(z.cpu().numpy(), y1)
    w = dev(c)
    cjt.cjt_inverse(plan, w, w)
    torch.cuda.synchronize()
    assert np.max(np.abs(w.cpu().numpy() - orc.inverse(c, a, b))) <= TOL * l1(c)


def test_execute_host_matches_device(cjt):
    N, a, b = 1024, -0.2, 0.4
    c = inputs.decaying_coefficients(N, 1.0, 4)
    plan = cjt.Plan(N, a, b)
    h = cjt.cjt_execute_host(plan, cjt.CJT_FWD, c)
    d = run_fwd(cjt, plan, c)
    assert np.array_equal(h, d)
    h = cjt.cjt_execute_host(plan, cjt.CJT_INV, c)
    d = run_inv(cjt, plan, c)
    assert np.array_equal(h, d)


def test_error_codes(cjt):
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, 1.6, 0.0)
    assert e.value.code == cjt.CJT_EDOMAIN
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(-1, 0.0, 0.0)
    assert e.value.code == cjt.CJT_EINVAL
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, 0.0, 0.0, M=21)
    assert e.value.code == cjt.CJT_EINVAL
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, 0.0, 0.0, grid=2)
    assert e.value.code == cjt.CJT_EINVAL
    p = cjt.Plan(64, 0.0, 0.0, directions=cjt.CJT_FWD)
    with pytest.raises(cjt.CJTError) as e:
        cjt.cjt_inverse(p, dev(np.zeros(65)))
    assert e.value.code == cjt.CJT_EDIRECTION


def test_identity_at_N0(cjt):
    p = cjt.Plan(0, 0.2, 0.1)
    assert run_fwd(cjt, p, np.array([2.5]))[0] == 2.5
    assert run_inv(cjt, p, np.array([-1.5]))[0] == -1.5


def default_grid(N):
    """The least G >= N of the forms 2^a, 3 2^a and 5 2^a."""
    G2 = 1 << (N - 1).bit_length() if N > 1 else 1
    G3, G5 = 3, 5
    while G3 < N:
        G3 <<= 1
    while G5 < N:
        G5 <<= 1
    return min(G2, G3, G5)


@pytest.mark.parametrize("grid", [0, 1, -1])
@pytest.mark.parametrize("alpha,beta", [(0.1, -0.3), (0.45, 0.45), (-0.5, 0.5)])
@pytest.mark.parametrize("N", [3, 5, 6, 7, 100, 1000, 1023, 1025, 3001, 10007])
def test_general_N_matches_oracle(cjt, orc, N, alpha, beta, grid):
    """N not a power of two: by default the evaluation runs on the least Lobatto grid G >= N
    of the forms 2^a, 3 2^a and 5 2^a (grid 0: transforms of lengths 3 2^b or 5 2^b take one
    radix-3 or radix-5 step), on the power-of-two grid with grid 1; on the paper's grid
    (grid -1) the DCT-I/DST-I sums go through Bluestein's chirp-z form unless N is 3 2^a or
    5 2^a."""
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 3 * N)
    plan = cjt.Plan(N, alpha, beta, grid=grid)
    info = plan.info()
    want = {0: default_grid(N), 1: 1 << (N - 1).bit_length(), -1: N}[grid]
    assert info["grid_fwd"] == want and info["grid_inv"] == 2 * info["grid_fwd"]
    assert info["fft_len_fwd"] == 2 * info["grid_fwd"] and info["fft_len_inv"] == 2 * info["grid_inv"]
    assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, alpha, beta))) <= TOL * l1(c)
    assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, alpha, beta))) <= TOL * l1(c)


@pytest.mark.parametrize("opts", [dict(rec_store=1), dict(M=13, ratio=0.05, seg_len=256), dict(use_asy=-1),
                                  dict(precision=2, rec_store=1), dict(precision=2, M=10), dict(M=3)])
@pytest.mark.parametrize("N", [1, 2, 4, 64, 1024])
def test_power_of_two_grid_forced(cjt, orc, N, opts):
    """grid = 1 on N that is already a power of two changes nothing; on N - 1 (one below
    a power of two) and N + 1 (just above) it evaluates on a grid of 2N rows or so."""
    for n in sorted({N, max(N - 1, 1), N + 1}):
        c = inputs.decaying_coefficients(n, 1.5, 4000 + n)
        plan = cjt.Plan(n, 0.2, -0.35, grid=1, **opts)
        assert plan.info()["grid_fwd"] == 1 << (n - 1).bit_length()
        assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, 0.2, -0.35))) <= TOL * l1(c), (n, opts)
        assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, 0.2, -0.35))) <= TOL * l1(c), (n, opts)


def test_power_of_two_grid_large(cjt, orc):
    """N = 40000 (grid 65536) and N = 70001 (grid 131072): the power-of-two grid against the
    paper's grid (Bluestein) and sampled oracle values; N = 3 * 2^20 + 1 plans on 2^22 by
    default (the smaller of 2^22 and 3 2^21)."""
    for N in (40000, 70001):
        c = inputs.decaying_coefficients(N, 1.5, 5000 + N)
        a, b = 0.3, -0.1
        pg = cjt.Plan(N, a, b, M=13, rec_store=1, grid=1)
        pb = cjt.Plan(N, a, b, M=13, rec_store=1, grid=-1)
        assert pg.info()["grid_fwd"] == 1 << (N - 1).bit_length() and pb.info()["grid_fwd"] == N
        fg = run_fwd(cjt, pg, c)
        assert np.max(np.abs(fg - run_fwd(cjt, pb, c))) <= TOL * l1(c)
        assert np.max(np.abs(run_inv(cjt, pg, c) - run_inv(cjt, pb, c))) <= TOL * l1(c)
        j = np.unique(np.concatenate([np.arange(0, 10), N - np.arange(0, 10), inputs.rng(12).integers(0, N + 1, 60)]))
        assert np.max(np.abs(orc.cheb_series(fg, j, N) - orc.jacobi_series(c, a, b, j, N))) <= TOL * l1(c)
        assert np.max(np.abs(run_inv(cjt, pg, fg) - c)) <= TOL * l1(c)
    big = cjt.Plan(3 * (1 << 20) + 1, 0.1, 0.2, directions=cjt.CJT_FWD, M=13)
    assert big.info()["grid_fwd"] == 1 << 22
    # and grids q 2^a at large size: N = 45000 plans on 49152 = 3 2^14 and N = 40000 on
    # 40960 = 5 2^13 by default
    for N, G in ((45000, 3 << 14), (40000, 5 << 13)):
        c = inputs.decaying_coefficients(N, 1.5, 5000 + N)
        pq = cjt.Plan(N, 0.3, -0.1, M=13, rec_store=1)
        p2 = cjt.Plan(N, 0.3, -0.1, M=13, rec_store=1, grid=1)
        assert pq.info()["grid_fwd"] == G and pq.info()["fft_len_inv"] == 4 * G
        assert np.max(np.abs(run_fwd(cjt, pq, c) - run_fwd(cjt, p2, c))) <= TOL * l1(c)
        assert np.max(np.abs(run_inv(cjt, pq, c) - run_inv(cjt, p2, c))) <= TOL * l1(c)
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(3 * (1 << 20) + 1, 0.1, 0.2, grid=-1)
    assert e.value.code == cjt.CJT_EUNSUPPORTED


# Mixed form (FP32 transforms of the asymptotic blocks, everything else FP64): stated bounds
MIXED_TOL_FWD = 1e-9
MIXED_TOL_INV = 1e-5


@pytest.mark.parametrize("N,M", [(1024, 7), (4096, 13), (3001, 10), (16384, 16), (65536, 16)])
def test_mixed_precision_within_stated_bound(cjt, orc, N, M):
    a, b = inputs.jacobi_parameters(inputs.BASE_SEED + 77 + N)
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 5 * N)
    plan = cjt.Plan(N, a, b, M=M, precision=cjt.CJT_MIXED)
    if N <= 16384:
        assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, a, b))) <= MIXED_TOL_FWD * l1(c)
        assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, a, b))) <= MIXED_TOL_INV * l1(c)
    # against the FP64 GPU form at any size
    p64 = cjt.Plan(N, a, b, M=M)
    assert np.max(np.abs(run_fwd(cjt, plan, c) - run_fwd(cjt, p64, c))) <= MIXED_TOL_FWD * l1(c)
    assert np.max(np.abs(run_inv(cjt, plan, c) - run_inv(cjt, p64, c))) <= MIXED_TOL_INV * l1(c)


@pytest.mark.parametrize("N", [1 << 16, 3001, 100])
def test_stored_recurrence_values(cjt, orc, N):
    """rec_store = 1 keeps the recurrence part of the matrix in device memory."""
    a, b = 0.3, -0.4
    c = inputs.decaying_coefficients(N, 1.5, 123)
    plan = cjt.Plan(N, a, b, rec_store=1, M=10)
    info = plan.info()
    # one double per recurrence step (padded to whole 32-row chunks)
    assert info["rec_store_bytes"] >= 8 * (info["rec_steps_fwd"] + info["rec_steps_inv"]) > 0
    assert np.max(np.abs(run_fwd(cjt, plan, c) - orc.forward(c, a, b))) <= TOL * l1(c)
    assert np.max(np.abs(run_inv(cjt, plan, c) - orc.inverse(c, a, b))) <= TOL * l1(c)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("overlap", [1, 2, 3])
@pytest.mark.parametrize("store", [0, 1])
def test_overlap_modes_are_bit_identical(cjt, orc, precision, overlap, store):
    """The option `overlap` only schedules the two concurrent chains of an execution:
    every mode gives the default plan's result bit for bit, on repeated executions, and
    the forward and inverse stay within the form's bound against the oracle."""
    N, a, b = 1 << 14, 0.1, -0.3
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 77)
    ref_plan = cjt.Plan(N, a, b, precision=precision, rec_store=store)
    plan = cjt.Plan(N, a, b, precision=precision, rec_store=store, overlap=overlap)
    assert ref_plan.info()["overlap"] == cjt.CJT_OVERLAP_ASY_FIRST
    assert plan.info()["overlap"] == overlap and plan.info()["nblk_fwd"] > 0 and plan.info()["nblk_inv"] > 0
    want_f, want_i = run_fwd(cjt, ref_plan, c), run_inv(cjt, ref_plan, c)
    for _ in range(2):
        assert np.array_equal(run_fwd(cjt, plan, c), want_f)
        assert np.array_equal(run_inv(cjt, plan, c), want_i)
    tol_f, tol_i = (1e-9, 1e-5) if precision == 1 else (TOL, TOL)
    assert np.max(np.abs(want_f - orc.forward(c, a, b))) <= tol_f * l1(c)
    assert np.max(np.abs(want_i - orc.inverse(c, a, b))) <= tol_i * l1(c)


def test_overlap_option_checked(cjt):
    for bad in (-1, 4):
        with pytest.raises(cjt.CJTError) as e:
            cjt.Plan(64, 0.1, -0.3, overlap=bad)
        assert e.value.code == cjt.CJT_EINVAL


@pytest.mark.parametrize("grid", [0, -1])
def test_golden_fixtures_exact_values(cjt, grid):
    """The CUDA path against the stored exact values at the paper's Fig. 1 parameters
    (alpha, beta) = (1/8, 3/8), N = 12 (tests/golden, written from exact rationals), on the
    power-of-two grid and on the paper's grid."""
    import os
    from fractions import Fraction
    here = os.path.join(os.path.dirname(__file__), "golden")
    for name, run in (("forward_exact_N12_a1o8_b3o8.txt", run_fwd), ("inverse_exact_N12_a1o8_b3o8.txt", run_inv)):
        meta, rows = {}, []
        for line in open(os.path.join(here, name)):
            line = line.strip()
            if line.startswith("#"):
                if ":" in line:
                    k, v = line[1:].split(":", 1)
                    meta[k.strip()] = v.strip()
            elif line:
                rows.append([Fraction(t) for t in line.split()])
        a, b = float(Fraction(meta["alpha"])), float(Fraction(meta["beta"]))
        c = np.array([float(r[0]) for r in rows])
        exact = np.array([float(r[1]) for r in rows])
        plan = cjt.Plan(len(c) - 1, a, b, grid=grid)
        assert np.max(np.abs(run(cjt, plan, c) - exact)) <= TOL * l1(c), name
        plan.close()

