"""CPU FP64 oracle of the PDHG + corner-push path (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The product (the CUDA library and its Python binding) never
imports it and shares no code with it; it exists to check the CUDA path.
Functions whose result no independent pin constrains say "parity unpinned" in
their docstring; every other function is pinned by the `-m "not gpu"` tests
(closed forms, brute-force vertex enumeration, constructed optima, HiGHS,
optimality conditions, published generator outputs).
"""
from .pdhg import (  # noqa: F401
    EQ, LE, GE, OPTIMAL, ITER_LIMIT, TIME_LIMIT, NUMERICAL, CORNER_DONE, CORNER_LIMIT,
    DEFAULTS, CORNER_DEFAULTS, Model, State, ruiz_pock_chambolle, power_iteration,
    project_box, project_dual_cone, primal_residual, dual_objective, evaluate, kkt_omega,
    pdhg_step, restart_check, initial_omega, setup, solve, run_iterations, unscale,
    splitmix64, splitmix64_uniform, corner_metrics, kkt_report, corner_model, corner_phase,
    dual_corner_model, dual_corner_phase,
)
