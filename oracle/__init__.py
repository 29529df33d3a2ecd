"""FP64 CPU oracle of the mixed-quadrature Shakhov lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline of the benchmark; never by the solver.
"""
