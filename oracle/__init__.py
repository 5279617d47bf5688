"""Oracle for the Q^k spectral-element fast-diagonalisation solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It is a plain, slow, FP64 CPU restatement of what the
paper's method computes (Liu, Shen, Zhang, "A simple GPU implementation of
spectral-element methods for solving 3D Poisson type equations on rectangular
domains", arXiv 2310.00226), written with numpy/scipy so that each step can be
checked against the paper by eye.  It shares no code with the CUDA library.

Every function cites the passage of the paper it follows.  Parity of every
function is pinned by ``tests/test_oracle_pins.py`` against values the paper or
the mathematics fix (closed forms, a dense assembled direct solve, Table 1, the
convergence order); no function here is "parity unpinned".
"""

from .sem import (  # noqa: F401
    gll_nodes_weights,
    legendre_p,
    diff_matrix,
    sem_1d,
    Sem1D,
    mode_product,
    fast_solve,
    fast_solve_x_line,
    apply_h,
    apply_weak,
    refined_solve,
    dense_solve,
    l2_error_table1,
    weak_matrix,
    schrodinger_solve,
    assembled_h3,
    bdf2_history,
    ch_explicit_term,
    ch_step,
)
from .tf32 import tf32_round, tf32_operand, fast_solve_rounded  # noqa: F401
