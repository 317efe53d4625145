"""Chebyshev exponential (paper Sec. 2.4, Eq. cheby and the recurrence after it).

The paper maps the imaginary interval i[-Lb, Lb], Lb = |lambda_max| t_max, to
[-1, 1] and uses P_0 = 1, P_1(l) = -i l / Lb, P_{k+1} = 2 l P_k / (i Lb) - P_{k-1},
with coefficients a_k from an FFT, then drops the highest coefficients while
their summed magnitude stays within a threshold (1e-6 in the paper).

Real form used here (an exact rewriting, checked in the tests): with
Q_k = i^k P_k, X = t L / Lb = sgn(t) L / lambda_max,
    Q_0 = v,  Q_1 = X v,  Q_{k+1} = 2 X Q_k + Q_{k-1},
    e^{tL} v = sum_k c_k Q_k,   c_k = a_k i^{-k}  (real).
t_max is taken equal to |t| for every call, so Lb = lambda_max |t|.
"""

import math

import numpy as np


def fft_size(Lb):
    return 1 << int(math.ceil(math.log2(Lb + 64.0)))


def chebyshev_coefficients_complex(Lb, n=None):
    """a_k of e^{i Lb y} = sum_k a_k T_k(y) on [-1, 1], by an FFT of samples at
    the Chebyshev-Lobatto points y_j = cos(pi j / n) (a DCT-I through the FFT of
    the even extension)."""
    n = fft_size(Lb) if n is None else n
    j = np.arange(n + 1)
    g = np.exp(1j * Lb * np.cos(np.pi * j / n))
    ext = np.concatenate([g, g[-2:0:-1]])                   # length 2n
    V = np.fft.fft(ext)[: n + 1]
    a = V / n
    a[0] /= 2.0
    a[n] /= 2.0
    return a


def chebyshev_coefficients(Lb, n=None):
    """Real coefficients c_k = a_k i^{-k} of the real recurrence."""
    a = chebyshev_coefficients_complex(Lb, n)
    k = np.arange(len(a))
    c = a * (1j) ** (-k)
    return c.real, c.imag


def truncation_degree(c, tol):
    """Smallest K with sum_{j > K} |c_j| <= tol: discard from the top while the
    discarded magnitude stays within the threshold (Sec. 2.4)."""
    K = len(c) - 1
    tail = 0.0
    while K > 0 and tail + abs(c[K]) <= tol:
        tail += abs(c[K])
        K -= 1
    return K


def truncated_coefficients(lam, t, tol):
    Lb = lam * abs(t)
    c, _ = chebyshev_coefficients(Lb)
    K = truncation_degree(c, tol)
    return c[: K + 1].copy()


def expL_apply(L, lam, t, v, tol):
    """e^{tL} v by the truncated Chebyshev series; L is a callable applying L."""
    if t == 0.0:
        return v.copy()
    c = truncated_coefficients(lam, t, tol)
    scale = math.copysign(1.0, t) / lam

    def X(w):
        return scale * L(w)

    q_prev = v
    out = c[0] * q_prev
    if len(c) == 1:
        return out
    q = X(v)
    out = out + c[1] * q
    for k in range(1, len(c) - 1):
        q_next = 2.0 * X(q) + q_prev
        out = out + c[k + 1] * q_next
        q_prev, q = q, q_next
    return out
