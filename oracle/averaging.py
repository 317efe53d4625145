"""Phase average by a weighted Riemann sum (paper Sec. 2.2).

Eq. vt_averaged weights the phase shift s by rho(s / T) with rho a smooth bump
supported on (-1/2, 1/2); Eq. vt_discretised replaces the integral by
sum_m w_m e^{-s_m L} N(e^{s_m L} U).

Readings (the printed bump and point set are garbled, so these are this
implementation's choices):
  * rho(x) = exp(-1 / (1/4 - x^2)) on |x| < 1/2, 0 elsewhere (the printed
    exponent has the wrong sign and would blow up at the ends);
  * the weights are normalised discretely, sum_m w_m = 1 (rho_0 cancels);
  * "midpoint" points: s_m = -T/2 + (m + 1/2) T / M, m = 0..M-1 (default);
    "closed" points: odd M = 2N + 1, s_k = k (T/2) / N, k = -N..N (the
    endpoints carry zero weight);
  * T = 0 gives N(U) itself (the delta-function limit the paper states).

The sum is the literal form: each shift has its own forward exponential, N,
and backward exponential, summed in shift order.
"""

import math

import numpy as np

QUAD_MIDPOINT = 0
QUAD_CLOSED = 1


def bump(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    inside = np.abs(x) < 0.5
    out[inside] = np.exp(-1.0 / (0.25 - x[inside] ** 2))
    return out


def shifts_and_weights(T, M, rule=QUAD_MIDPOINT):
    if M < 1:
        raise ValueError("M must be >= 1")
    if rule == QUAD_MIDPOINT:
        s = -0.5 * T + (np.arange(M) + 0.5) * T / M
    elif rule == QUAD_CLOSED:
        if M % 2 == 0 or M < 3:
            raise ValueError("closed rule needs odd M >= 3")
        Nh = (M - 1) // 2
        s = np.arange(-Nh, Nh + 1) * (0.5 * T) / Nh
    else:
        raise ValueError("unknown rule")
    if T == 0.0:
        return np.zeros(M), np.full(M, 1.0 / M)
    rho = bump(s / T)
    return s, rho / rho.sum()


def averaged_rhs(model, T, M, U, rule=QUAD_MIDPOINT):
    """<e^{-Ls} N(e^{Ls} U)>_s, literal per-shift form (Eq. vt_discretised)."""
    if T == 0.0:
        return model.N(U)
    s, w = shifts_and_weights(T, M, rule)
    out = np.zeros_like(U)
    for m in range(M):
        if w[m] == 0.0:
            continue
        V = model.expL(s[m], U)
        n = model.N(V)
        out += w[m] * model.expL(-s[m], n)
    return out


def averaged_rhs_group(model, T, M, m0, m1, U, rule=QUAD_MIDPOINT):
    """The terms m0 <= m < m1 of the M-point sum, with the whole rule's weights
    (the paper distributes the independent terms over process groups and
    reduces their partial sums once, Sec. 2.5)."""
    s, w = shifts_and_weights(T, M, rule)
    if T == 0.0:
        return (m1 - m0) / M * model.N(U)
    out = np.zeros_like(U)
    for m in range(m0, m1):
        if w[m] == 0.0:
            continue
        out += w[m] * model.expL(-s[m], model.N(model.expL(s[m], U)))
    return out


def averaged_rhs_marching(model, T, M, U, rule=QUAD_MIDPOINT):
    """The same sum by shift marching: the shifts are equally spaced, so with
    ds_m = s_{m+1} - s_m every shifted state follows from the previous one,
        V_0 = e^{s_0 L} U,   V_{m+1} = e^{ds_m L} V_m,
    and the backward maps nest (Horner),
        H_{M-1} = w_{M-1} N(V_{M-1}),  H_m = w_m N(V_m) + e^{-ds_m L} H_{m+1},
        sum = e^{-s_0 L} H_0.
    Each short exponential is truncated by the same tail rule (Sec. 2.4), so
    the result differs from the direct sum by the truncation errors of the
    extra exponentials; with a tight tail threshold the two agree."""
    if T == 0.0:
        return model.N(U)
    s, w = shifts_and_weights(T, M, rule)
    V = [model.expL(s[0], U)]
    for m in range(1, M):
        V.append(model.expL(s[m] - s[m - 1], V[-1]))
    H = w[M - 1] * model.N(V[M - 1]) if w[M - 1] != 0.0 else np.zeros_like(U)
    for m in range(M - 2, -1, -1):
        H = model.expL(-(s[m + 1] - s[m]), H)
        if w[m] != 0.0:
            H = H + w[m] * model.N(V[m])
    return model.expL(-s[0], H)


def averaged_rhs_term(model, s, U):
    """One term e^{-sL} N(e^{sL} U) of the sum (unweighted)."""
    return model.expL(-s, model.N(model.expL(s, U)))


def weights_sum(T, M, rule=QUAD_MIDPOINT):
    return float(math.fsum(shifts_and_weights(T, M, rule)[1]))
