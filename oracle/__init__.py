"""CPU oracle for the time-domain Casimir method (arXiv:0906.5170).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu-baseline leg of bench.py may import this package.  The product path
(paper_0906_5170_gb300) never imports it, and it never imports the product.

Plain, slow, FP64: numpy for the set-up (rasterisation, basis, interpolation,
g(t)), plain C loops (yee_oracle.c) for the leapfrog itself.
"""
from .casimir_oracle import (  # noqa: F401
    build_library, build_all, img_minus_t, g_weights, enumerate_sims, run_sim, force,
    evolve, grid_setup, face_pixels, harmonic, interp_weights, run_vectors,
    is_cyl, cyl_site_weight, E_OFF, H_OFF, lorentz_poles, MAX_POLES,
)
