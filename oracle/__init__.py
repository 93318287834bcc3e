"""FP64 CPU oracle for the lifted PDHG solver (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path.  See ``lift_oracle.c`` for what each function
computes and which passage of arXiv 1512.01383 it follows.
"""
from .oracle import (  # noqa: F401
    QUAD, TRUNC, PL, PERIODIC, Problem, State, build, conj, lifted_conj, proj_epi, biconj,
    rho, grad, div, steps, pdhg, unlift, monotone_proj, energy, rof_direct,
    rof_energy, labels, unrolled_grad, movement, pdhg_adaptive, grad3, div3, rof_direct3,
    rof_energy3, half_step, pdhg_averaged, solve_restarted,
)
