"""CPU oracle for the lattice Boltzmann hot path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package.  The product library never does, and nothing here imports the product.
``lbm_oracle.c`` is the plain FP64 implementation; ``single_cell.py`` is an independent NumPy
restatement of the single-cell collision used to cross-check it.
"""
from .oracle import (  # noqa: F401
    FLUID, NOSLIP, VELOCITY, PRESSURE, PERIODIC, ZOUHE_VELOCITY, ZOUHE_PRESSURE, SRT, TRT, MRT, CUMULANT, mrt_matrix, mrt_rates,
    cumulants, cumulants_to_f, refine_fine_params, refine_slab_flags, refine_init, refine_run,
    OracleParams, build_oracle, lattice, omega_minus, equilibrium, collide_cell,
    init, run, stream, macroscopic, diagnostics, set_threads, get_threads,
    NO_CLOSURE, SMAGORINSKY, MLP, collide_closure,
)
