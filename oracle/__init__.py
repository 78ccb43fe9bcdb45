"""Test infrastructure: the CPU oracle for persistent homology of cubical images.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
from .oracle import (  # noqa: F401
    build,
    persistence,
    persistence_f64,
    num_cells,
    cell_value,
    cell_vertices,
    argmax_vertex,
    gradient,
    filtration,
    brute_force_pairs,
    brute_force_rank_diagram,
    h0_1d_brute_force,
    euler_characteristic,
    pair_table,
    lifetime_image,
    persistent_histogram_image,
)
