"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This package builds *problem data only*: the polynomial trajectory problems
(objective, inequality and equality polynomials per clique, Definition 1 /
eq. (1)) and the random symmetric matrices of the PSD-projection microbench.
It contains none of the relaxation, ADMM or projection arithmetic; both the
oracle and the CUDA path read what it produces.
"""
from .poly import Poly
from .problems import (BASE_SEED, Problem, Clique, toy_problem, pendulum_problem, paper_pendulum_problem,
                       paper_landing_problem, paper_flying_robot_problem, paper_car_backin_problem,
                       cartpole_problem, rigid_body_problem, problem_batch, SERVING_MIX, mixed_request,
                       poisson_arrivals)
from .psd_bench import psd_microbench, known_spectrum_blocks

__all__ = ["BASE_SEED", "Poly", "Problem", "Clique", "toy_problem", "pendulum_problem", "paper_pendulum_problem",
           "paper_landing_problem", "paper_flying_robot_problem", "paper_car_backin_problem",
           "cartpole_problem", "rigid_body_problem", "problem_batch", "SERVING_MIX", "mixed_request", "poisson_arrivals",
           "psd_microbench", "known_spectrum_blocks"]
