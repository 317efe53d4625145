"""Averaged Lawson RK4 (paper Sec. 2.3, Eqs. stage1_c, stage2s, stage3s, stage4).

With <.> the phase average of the model (N-bar) and E(t) = e^{tL}:
  U1      = U^n + dt/2 N-bar(U^n)
  U2      = E(dt/2) U^n + dt/2 N-bar(E(dt/2) U1)
  U3      = E(dt/2) U^n + dt   N-bar(U2)
  U^{n+1} = E(dt) U^n + dt/6 [ E(dt) N-bar(U^n) + 2 E(dt/2) N-bar(E(dt/2) U1)
                              + 2 E(dt/2) N-bar(U2) + N-bar(E(dt/2) U3) ]
(the exponentials inside the brackets commute with the average, so
<e^{-Ls} N(e^{L dt/2} e^{Ls} U1)> = N-bar(E(dt/2) U1)).  Written here term by
term, each exponential applied separately as printed.
"""


def lawson_rk4_step(model, dt, T, M, U, rule=0):
    avg = lambda V: model.averaged_rhs(T, M, V, rule)  # noqa: E731
    Eh = lambda V: model.expL(0.5 * dt, V)              # noqa: E731
    E = lambda V: model.expL(dt, V)                     # noqa: E731
    k1 = avg(U)
    U1 = U + 0.5 * dt * k1
    EhU = Eh(U)
    k2 = avg(Eh(U1))
    U2 = EhU + 0.5 * dt * k2
    k3 = avg(U2)
    U3 = EhU + dt * k3
    k4 = avg(Eh(U3))
    return E(U) + (dt / 6.0) * (E(k1) + 2.0 * Eh(k2) + 2.0 * Eh(k3) + k4)
