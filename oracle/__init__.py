"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle of the two-phase lattice Boltzmann step.

Plain, slow and meant to be checked by eye against Yu, Li & Wen, "Modified curved boundary
scheme for two-phase lattice Boltzmann simulations" (arXiv:1908.09235).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  It shares no code with the CUDA library.

Functions whose result is pinned to something other than the oracle itself are listed in
``tests/test_oracle_pins.py``; every public function here has at least one such pin.
"""
from .binding import (  # noqa: F401
    HBB, FH, MLS, BOUZIDI_L, BOUZIDI_Q, ZHAO_YONG, MOD_A, MOD_B, BAO, BOUZIDI_L_A,
    EOS_NONE, EOS_EXP, EOS_CS, SCHEME_NAMES,
    OracleSim, feq, guo, collide_node, psi, cs_pressure, force_from_psi, cs_critical,
    cs_coexistence, build_oracle, library_path, num_threads,
)
