"""The FP32 transform error constant of the mixed form's stated bound, checked on a NumPy model
of the transform the mixed form runs.

The mixed form bounds each output of an FP32 transform of length L by eps_F * sum_n |z_n|, with
eps_F = u (3 ceil(log2 L) + 8) and u = 2^-24 (the per-plan bound of `cjt_error_bound` builds
on it).  The model below follows the transform's structure step by step in complex64
arithmetic, each operation rounded to FP32:
  * radix-4 decimation-in-frequency stages, after one radix-2 stage when log2 L is odd, with
    the twiddles omega_span^j rounded to FP32;
  * above the one-pass limit, the four-step split L = L1 L2 (column transforms of length L1,
    the twiddle omega_L^{n2 k1} rounded to FP32, row transforms of length L2);
  * for L = q 2^a (q = 3, 5), one q-point DFT step over x[n2 + L2 n1] with FP32 constants and
    the twiddle omega_L^{k1 n2}, then q transforms of length L2 whose outputs go to
    X[k1 + q k2];
  * the input rounded to FP32 first (the pack's rounding).
Its outputs are compared with the exact DFT (complex128) of the unrounded input.  The pin:
every output's error stays below eps_F * ||z||_1, for random inputs and for inputs whose phases
are aligned with one output (the case the l1 bound is written for).  The bound is not vacuous:
aligned inputs reach a few percent of it.
"""
import numpy as np
import pytest

U = 2.0 ** -24
C64 = np.complex64


def eps_f(L):
    return U * (3 * int(np.ceil(np.log2(L))) + 8)


def _tw(n, k):
    """omega_n^k = exp(-2 pi i k / n), rounded to FP32 from a double value."""
    return np.exp(-2j * np.pi * (np.asarray(k) % n) / n).astype(C64)


def dif_positions(L):
    """Output slot of each frequency k after the radix-2/radix-4 DIF stages: a first stage of
    radix r over span L leaves frequency k = i + r k' in sub-block i at the slot of k' there."""
    lg = int(np.log2(L))
    radices = ([2] if lg % 2 else []) + [4] * (lg // 2)
    k = np.arange(L)
    pos = np.zeros(L, dtype=np.int64)
    span = L
    for r in radices:
        span //= r
        pos += (k % r) * span
        k = k // r
    return pos


def r4_dif_f32(x):
    """Batched (rows) FP32 power-of-two DIF transform along the last axis, natural order."""
    x = np.array(x, dtype=C64, copy=True)
    B, L = x.shape
    lg = int(np.log2(L))
    span = L
    if lg % 2:
        h = span // 2
        v = x.reshape(B, -1, span)
        a, b = v[:, :, :h].copy(), v[:, :, h:].copy()
        v[:, :, :h] = a + b
        v[:, :, h:] = (a - b) * _tw(span, np.arange(h))
        span = h
    mi = C64(-1j)
    while span >= 4:
        q = span // 4
        v = x.reshape(B, -1, span)
        a0, a1, a2, a3 = (v[:, :, i * q:(i + 1) * q].copy() for i in range(4))
        j = np.arange(q)
        t0, t1, t2, t3 = a0 + a2, a0 - a2, a1 + a3, (a1 - a3) * mi
        v[:, :, :q] = t0 + t2
        v[:, :, q:2 * q] = (t1 + t3) * _tw(span, j)
        v[:, :, 2 * q:3 * q] = (t0 - t2) * _tw(span, 2 * j)
        v[:, :, 3 * q:] = (t1 - t3) * _tw(span, 3 * j)
        span = q
    return x[:, dif_positions(L)]


def fft_pow2_f32(x, one_pass_log2=12):
    """Batched FP32 transform of length 2^b: one pass up to 2^one_pass_log2, else four-step."""
    B, L = x.shape
    lg = int(np.log2(L))
    if lg <= one_pass_log2:
        return r4_dif_f32(x)
    L1 = 1 << (lg // 2)
    L2 = L // L1
    a = x.reshape(B, L1, L2).transpose(0, 2, 1).reshape(B * L2, L1)       # x[L2 n1 + n2] over n1
    A = r4_dif_f32(a).reshape(B, L2, L1)                                   # A[n2, k1]
    A = A * _tw(L, np.outer(np.arange(L2), np.arange(L1)))                 # omega_L^{n2 k1}
    X = r4_dif_f32(A.transpose(0, 2, 1).reshape(B * L1, L2)).reshape(B, L1, L2)   # X[k1, k2]
    return X.transpose(0, 2, 1).reshape(B, L)                              # k = k1 + L1 k2


def fft_f32(z, q=1, one_pass_log2=12):
    """FP32 model of a transform of length L = q 2^a (q = 1, 3 or 5) of one vector z."""
    x = np.asarray(z).astype(C64)[None, :]                                 # the pack's rounding
    if q == 1:
        return fft_pow2_f32(x, one_pass_log2)[0]
    L = x.shape[1]
    L2 = L // q
    v = x.reshape(q, L2)                                                   # v[n1, n2] = x[n2 + L2 n1]
    cq = _tw(q, np.outer(np.arange(q), np.arange(q)))                      # omega_q^{n1 k1}, FP32
    y = np.zeros((q, L2), dtype=C64)
    for k1 in range(q):
        acc = v[0] * cq[0, k1]
        for n1 in range(1, q):
            acc = acc + v[n1] * cq[n1, k1]
        y[k1] = acc * _tw(L, k1 * np.arange(L2))                           # omega_L^{k1 n2}
    Y = fft_pow2_f32(y, one_pass_log2)                                     # Y[k1, k2]
    return Y.T.reshape(L)                                                  # X[k1 + q k2]


def _inputs(L, seed):
    rng = np.random.default_rng(seed)
    out = [rng.standard_normal(L) + 1j * rng.standard_normal(L),
           rng.uniform(0.0, 1.0, L) * np.exp(2j * np.pi * rng.random(L))]
    for _ in range(3):                       # phases aligned with one output k0
        k0 = int(rng.integers(L))
        out.append(rng.uniform(0.5, 1.0, L) * np.exp(2j * np.pi * k0 * np.arange(L) / L))
    return out


CASES = [(1, 1 << b) for b in range(2, 15)] + [(3, 3 << 4), (3, 3 << 10), (3, 3 << 13), (5, 5 << 4),
                                                (5, 5 << 10), (5, 5 << 12)]


def test_model_is_the_dft():
    """The model computes the DFT: its FP32 outputs, in natural order, agree with numpy's
    FFT to FP32 accuracy."""
    for q, L in [(1, 64), (1, 128), (1, 1 << 13), (3, 3 << 6), (5, 5 << 5)]:
        z = _inputs(L, 7)[0]
        got = fft_f32(z, q).astype(np.complex128)
        want = np.fft.fft(z)
        assert np.abs(got - want).max() <= 1e-4 * np.abs(z).sum() / np.sqrt(L)


@pytest.mark.parametrize("q,L", CASES, ids=lambda v: str(v))
def test_fp32_transform_error_within_eps_f(q, L):
    worst = 0.0
    for t, z in enumerate(_inputs(L, 1000 + L + q)):
        err = np.abs(fft_f32(z, q).astype(np.complex128) - np.fft.fft(z)).max()
        ratio = err / (eps_f(L) * np.abs(z).sum())
        assert ratio <= 1.0, (q, L, t, ratio)
        worst = max(worst, ratio)
    assert worst > 1e-4        # errors of the order the bound describes were produced


def test_eps_f_is_not_vacuous():
    """Inputs aligned with one output reach a few percent of eps_F ||z||_1 (so the constant
    is within two orders of magnitude of the worst case the model produces)."""
    worst = 0.0
    for q, L in CASES:
        for z in _inputs(L, 2000 + L + q)[2:]:
            err = np.abs(fft_f32(z, q).astype(np.complex128) - np.fft.fft(z)).max()
            worst = max(worst, err / (eps_f(L) * np.abs(z).sum()))
    assert 0.02 < worst <= 1.0
