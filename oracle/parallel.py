"""The oracle's literal averaged sum with its terms spread over host processes.

Test and benchmark infrastructure, like the rest of oracle/: only tests/,
the smoke check and the benchmark's CPU-baseline leg use it; the library never
does.

Each term e^{-s_m L} N(e^{s_m L} U) of Eq. vt_discretised (Sec. 2.2) is
independent of the others (the paper's own parallel step, Sec. 2.5, last
paragraph).  Worker processes (started with "spawn", so they inherit no CUDA
state) each build one OracleModel and evaluate whole terms with
averaging.averaged_rhs_term; the parent adds w_m * term_m in shift order
m = 0..M-1, exactly as averaging.averaged_rhs does, so the result is bitwise
the sequential oracle's.
"""

import dataclasses
import multiprocessing as mp
import os

import numpy as np

from . import averaging
from .model import OracleModel, OracleParams

_M = None


def _init(params, nice):
    global _M
    if nice:
        try:
            os.nice(nice)
        except OSError:
            pass
    _M = OracleModel(OracleParams(**params))


def _term(args):
    s, U = args
    return averaging.averaged_rhs_term(_M, s, U)


def _norms(V):
    u, e = _M.ops.split(V)
    return float(np.sqrt(u @ (_M.ops.M1 @ u))), float(np.sqrt(e @ (_M.ops.M2 @ e)))


class OraclePool:
    """A pool of spawned processes holding one oracle model each."""

    def __init__(self, params: OracleParams, workers=None, nice=0):
        self.params = params
        self.workers = workers or max(1, os.cpu_count() or 1)
        ctx = mp.get_context("spawn")
        # one BLAS thread per worker: the children read these when numpy loads
        keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            self.pool = ctx.Pool(self.workers, initializer=_init,
                                 initargs=(dataclasses.asdict(params), nice))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def degree(self, t):
        from . import expo
        return len(expo.truncated_coefficients(self.params.lambda_max, t, self.params.cheb_tol)) - 1

    def averaged_rhs(self, T, M, U, rule=None):
        """sum_m w_m e^{-s_m L} N(e^{s_m L} U), literal form, terms in parallel."""
        rule = self.params.quad_rule if rule is None else rule
        s, w = averaging.shifts_and_weights(T, M, rule)
        todo = [m for m in range(M) if w[m] != 0.0]
        if T == 0.0 or not todo:
            raise ValueError("T = 0 (a single N) needs no pool")
        # longest chains first so that the workers finish together
        order = sorted(todo, key=lambda m: -self.degree(s[m]))
        terms = dict(zip(order, self.pool.map(_term, [(s[m], U) for m in order], chunksize=1)))
        out = np.zeros_like(U)
        for m in todo:
            out += w[m] * terms[m]
        return out

    def norms(self, V):
        """(||u||_M1, ||eta||_M2) of one state (computed in a worker)."""
        return self.pool.apply(_norms, (V,))

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()
