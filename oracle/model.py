"""One oracle instance: mesh + operators + exponential + average + timestep."""

from dataclasses import dataclass

from . import averaging, expo, spectrum, timestep
from .mesh import build_mesh
from .operators import UPWIND_STANDARD, Operators


@dataclass
class OracleParams:
    refinement: int = 3
    radius: float = 6.37122e6
    omega: float = 7.292e-5
    g: float = 9.80616
    H: float = 5000.0
    cheb_tol: float = 1e-6
    lambda_max: float = 0.0      # 0 -> power iteration
    quad_rule: int = averaging.QUAD_MIDPOINT
    upwind: int = UPWIND_STANDARD
    geometry_degree: int = 1     # 1 flat cells, 3 the piecewise cubic surface of Sec. 3


class OracleModel:
    def __init__(self, params: OracleParams):
        self.p = params
        self.mesh = build_mesh(params.refinement, params.radius)
        self.ops = Operators(self.mesh, params.g, params.H, params.omega, params.radius, params.upwind,
                             geometry_degree=params.geometry_degree)
        self.n_u, self.n_eta, self.n = self.ops.n_u, self.ops.n_eta, self.ops.n
        self.lam = params.lambda_max if params.lambda_max > 0 else spectrum.power_iteration(self.ops)

    def L(self, U):
        return self.ops.L(U)

    def N(self, U):
        return self.ops.N(U)

    def expL(self, t, U):
        return expo.expL_apply(self.ops.L, self.lam, t, U, self.p.cheb_tol)

    def averaged_rhs(self, T, M, U, rule=None):
        return averaging.averaged_rhs(self, T, M, U, self.p.quad_rule if rule is None else rule)

    def timestep(self, dt, T, M, U, nsteps=1):
        for _ in range(nsteps):
            U = timestep.lawson_rk4_step(self, dt, T, M, U, self.p.quad_rule)
        return U

    def degree(self, t):
        return len(expo.truncated_coefficients(self.lam, t, self.p.cheb_tol)) - 1
