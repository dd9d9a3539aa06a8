"""GPU parity of the reduced-complexity parameter cases (App. B) against the CPU oracle.

* alpha = beta = lambda - 1/2 (App. B.1): plans use the ultraspherical formula by default
  (one cosine per term in u_m, v_m; its own coefficients, remainder bound and n_M).
  Hahn's formula, forced, gives the same transform to rounding.
* alpha or beta = +-1/2 (App. B.2-B.3): each term of Hahn's formula is one cosine.
The tolerance is the library's FP64 bound max |c_gpu - c_oracle| <= 1e-12 ||c||_1.
"""
import math

import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
DIAG = [(0.0, 0.0), (0.3, 0.3), (-0.3, -0.3), (0.45, 0.45), (-0.45, -0.45), (0.05, 0.05)]
COLLAPSE = [(0.5, 0.2), (0.3, 0.5), (-0.5, 0.1), (0.2, -0.5), (0.5, -0.45)]


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


def run(cjt, plan, c, direction):
    fn = cjt.cjt_forward if direction == cjt.CJT_FWD else cjt.cjt_inverse
    y = fn(plan, dev(c))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def check(cjt, orc, plan, c, a, b):
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, a, b))) <= TOL * l1(c), plan.info()
    assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, a, b))) <= TOL * l1(c), plan.info()


@pytest.mark.parametrize("a,b", DIAG)
@pytest.mark.parametrize("N", [2, 8, 64, 1024, 4096])
def test_ultraspherical_matches_oracle(cjt, orc, N, a, b):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 17 * N)
    plan = cjt.Plan(N, a, b)
    assert plan.info()["expansion"] == cjt.CJT_EXPANSION_ULTRASPHERICAL
    check(cjt, orc, plan, c, a, b)


@pytest.mark.parametrize("opts", [dict(M=3), dict(M=7), dict(M=13), dict(M=20), dict(rec_store=1),
                                  dict(M=13, rec_store=1, seg_len=256, ratio=0.05), dict(use_asy=-1),
                                  dict(precision=2, rec_store=1, M=13), dict(precision=2, M=10),
                                  dict(expansion=1), dict(expansion=1, rec_store=1, M=13)])
def test_ultraspherical_options(cjt, orc, opts):
    N, a = 4096, 0.3
    c = inputs.decaying_coefficients(N, 1.5, 4242)
    plan = cjt.Plan(N, a, a, **opts)
    check(cjt, orc, plan, c, a, a)


@pytest.mark.parametrize("N", [3, 1000, 3001])
def test_ultraspherical_general_N(cjt, orc, N):
    a = 0.2
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 5 * N)
    check(cjt, orc, cjt.Plan(N, a, a, rec_store=1), c, a, a)


@pytest.mark.parametrize("a,b", COLLAPSE)
@pytest.mark.parametrize("N", [64, 1024, 4096])
def test_collapsed_terms_match_oracle(cjt, orc, N, a, b):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 23 * N)
    plan = cjt.Plan(N, a, b, M=10)
    assert plan.info()["expansion"] == cjt.CJT_EXPANSION_HAHN
    check(cjt, orc, plan, c, a, b)


@pytest.mark.parametrize("a", [0.0, 0.25, -0.4])
def test_ultraspherical_full_size(cjt, orc, a):
    """N = 2^16: the ultraspherical and Hahn plans agree within the bound, the forward result
    matches sampled oracle values, and the round trip closes."""
    N = 1 << 16
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + 77)
    pu = cjt.Plan(N, a, a, M=13, rec_store=1)
    ph = cjt.Plan(N, a, a, M=13, rec_store=1, expansion=cjt.CJT_EXPANSION_HAHN)
    assert pu.info()["expansion"] == cjt.CJT_EXPANSION_ULTRASPHERICAL
    assert ph.info()["expansion"] == cjt.CJT_EXPANSION_HAHN
    fu = run(cjt, pu, c, cjt.CJT_FWD)
    assert np.max(np.abs(fu - run(cjt, ph, c, cjt.CJT_FWD))) <= TOL * l1(c)
    iu = run(cjt, pu, c, cjt.CJT_INV)
    assert np.max(np.abs(iu - run(cjt, ph, c, cjt.CJT_INV))) <= TOL * l1(c)
    j = np.unique(np.concatenate([np.arange(0, 20), N - np.arange(0, 20), inputs.rng(9).integers(0, N + 1, 200)]))
    assert np.max(np.abs(orc.cheb_series(fu, j, N) - orc.jacobi_series(c, a, a, j, N))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, pu, fu, cjt.CJT_INV) - c)) <= TOL * l1(c)


def test_ultraspherical_n_M_is_the_closed_form(cjt):
    """n_M of an ultraspherical plan is App. B.1's closed form; Hahn's is Sec. 2.2's."""
    eps = 2.0 ** -52
    for lam in (0.2, 0.5, 0.8):
        for M in (5, 7, 13):
            a = lam - 0.5
            poch = math.prod((lam + k) * (1 - lam + k) for k in range(M))
            nM = math.floor((eps * math.sqrt(math.pi) * 2 ** M * math.factorial(M) /
                             (2 ** (lam + 1) * poch)) ** (-1.0 / (M + 0.5)))
            info = cjt.Plan(4096, a, a, M=M).info()
            assert abs(info["n_M"] - nM) <= 1, (lam, M, info["n_M"], nM)


def test_shifted_diagonal(cjt, orc):
    """(1.2, 1.2) runs the ultraspherical plan at (0.2, 0.2) with both unit shifts (Sec. 1.2)."""
    N, a = 1024, 1.2
    c = inputs.decaying_coefficients(N, 1.0, 31)
    plan = cjt.Plan(N, a, a)
    info = plan.info()
    assert info["expansion"] == cjt.CJT_EXPANSION_ULTRASPHERICAL and info["shift_alpha"] == info["shift_beta"] == 1
    check(cjt, orc, plan, c, a, a)


def test_expansion_option_errors(cjt):
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, 0.1, 0.2, expansion=cjt.CJT_EXPANSION_ULTRASPHERICAL)
    assert e.value.code == cjt.CJT_EINVAL
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, 0.1, 0.1, expansion=3)
    assert e.value.code == cjt.CJT_EINVAL
    # corners: one exact term whichever formula is asked for
    for a in (0.5, -0.5):
        info = cjt.Plan(256, a, a, expansion=cjt.CJT_EXPANSION_ULTRASPHERICAL).info()
        assert info["M"] == 1


# ---------------------------------------------------------------------------
# parity fold: alpha = beta with stored recurrence values (P_n(-x) = (-1)^n P_n(x))
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("a", [0.0, 0.3, -0.45, 0.5, -0.5])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 7, 64, 1023, 1024, 4096])
def test_parity_fold_matches_oracle(cjt, orc, N, a, prec):
    c = inputs.decaying_coefficients(N, 1.0, inputs.BASE_SEED + 29 * N)
    plan = cjt.Plan(N, a, a, rec_store=1, precision=prec)
    assert plan.info()["parity_fold"] == 1
    check(cjt, orc, plan, c, a, a)


@pytest.mark.parametrize("opts", [dict(use_asy=-1), dict(seg_len=32), dict(M=13, ratio=0.05, seg_len=256),
                                  dict(expansion=1), dict(M=3), dict(precision=2, use_asy=-1, seg_len=64),
                                  dict(precision=1)])
def test_parity_fold_options(cjt, orc, opts):
    N, a = 3001 if opts.get("seg_len") == 32 else 4096, -0.2
    c = inputs.decaying_coefficients(N, 1.5, 777)
    plan = cjt.Plan(N, a, a, rec_store=1, **opts)
    assert plan.info()["parity_fold"] == 1
    if opts.get("precision") == 1:   # mixed form: its stated bounds (forward 1e-9, inverse 1e-5)
        assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_FWD) - orc.forward(c, a, a))) <= 1e-9 * l1(c)
        assert np.max(np.abs(run(cjt, plan, c, cjt.CJT_INV) - orc.inverse(c, a, a))) <= 1e-5 * l1(c)
    else:
        check(cjt, orc, plan, c, a, a)


def test_parity_fold_halves_the_stored_values(cjt):
    """The folded plan stores (and runs) about half the recurrence of the same plan without
    the fold (alpha = beta + 1e-9: the same partition to within a row or two)."""
    N, a = 1 << 14, 0.25
    pf = cjt.Plan(N, a, a, rec_store=1, M=10, expansion=cjt.CJT_EXPANSION_HAHN)
    pn = cjt.Plan(N, a, a + 1e-9, rec_store=1, M=10)
    fi, ni = pf.info(), pn.info()
    assert fi["parity_fold"] == 1 and ni["parity_fold"] == 0
    for key in ("rec_store_bytes", "rec_steps_fwd", "rec_steps_inv"):
        assert 0.45 * ni[key] <= fi[key] <= 0.55 * ni[key], (key, fi[key], ni[key])
    assert cjt.Plan(64, a, a).info()["parity_fold"] == 0   # only with stored values


@pytest.mark.parametrize("prec", [0, 2])
def test_parity_fold_full_size(cjt, orc, prec):
    """Legendre (alpha = beta = 0) at N = 2^18: the folded plan against the unfolded one (the
    recurrence at execution), sampled oracle values and the round trip."""
    N, a = 1 << 18, 0.0
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED + 88)
    pf = cjt.Plan(N, a, a, M=13, rec_store=1, seg_len=1024, precision=prec)
    p0 = cjt.Plan(N, a, a, M=13, seg_len=1024)
    assert pf.info()["parity_fold"] == 1 and p0.info()["parity_fold"] == 0
    ff = run(cjt, pf, c, cjt.CJT_FWD)
    assert np.max(np.abs(ff - run(cjt, p0, c, cjt.CJT_FWD))) <= TOL * l1(c)
    fi = run(cjt, pf, c, cjt.CJT_INV)
    assert np.max(np.abs(fi - run(cjt, p0, c, cjt.CJT_INV))) <= TOL * l1(c)
    j = np.unique(np.concatenate([np.arange(0, 20), N - np.arange(0, 20), inputs.rng(10).integers(0, N + 1, 100)]))
    assert np.max(np.abs(orc.cheb_series(ff, j, N) - orc.jacobi_series(c, a, a, j, N))) <= TOL * l1(c)
    assert np.max(np.abs(run(cjt, pf, ff, cjt.CJT_INV) - c)) <= TOL * l1(c)
