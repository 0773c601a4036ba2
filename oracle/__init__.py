"""FP64 CPU oracle for multigrid ISDF and the THC exact-exchange build.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (the CUDA library and its Python binding) never imports, links or
calls it, and the two share no code: the oracle is written from the paper's
equations in plain NumPy/SciPy, slowly and literally, so that a reader can check
it against the paper by eye.

Parity status of each function is stated in its docstring; a function with no
independent pin says "parity unpinned".
"""
from .isdf import (  # noqa: F401
    expand_functions,
    level_sets,
    basis_on_level,
    basis_direct,
    initial_diagonal,
    select_points,
    fit,
    coulomb,
    exchange,
    run,
    run_sinc,
    coarse_points,
    run_local,
    local_grid,
    local_radius,
    PIVOT_SHIFT,
)
from .nofit import nofit_exchange, brute_exchange, brute_exchange_local  # noqa: F401
