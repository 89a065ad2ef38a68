"""Seeded synthetic problem generators shared by the oracle, the tests and the bench.

This package builds problem *data* only (A, b, bounds, planted solutions) and holds
none of the solver's arithmetic: no gradient, best response, step or objective.

Layout convention used everywhere: the m x n matrix A is stored column-major, i.e.
as an array ``At`` of shape (n, lda) whose row j is column a_j of A (rows m..lda-1
of each column are zero padding).
"""

from .problems import (  # noqa: F401
    nesterov_lasso,
    nesterov_lasso_torch,
    random_lasso,
    ncquad_problem,
    dc_problem,
    liu_wright_lasso,
    liu_wright_lasso_torch,
    dc_problem_torch,
    ncquad_problem_torch,
    pad_lda,
    validation_rows,
    validation_rows_torch,
)
