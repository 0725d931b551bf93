"""FP64 CPU oracle of the relativistic lattice Boltzmann model (arXiv:1301.3423).

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the GPU library is checked against.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.  It
shares no code with the GPU path.

``core``        serial C step (pull, moments, Landau matching, projected equilibrium, collision)
                behind ctypes, the explicit App. B equilibrium as a cross-check, and the
                lattice-table reader;
``projection``  the equilibrium as an explicit Gram-Schmidt projection in numpy, an independent
                route to the same f_i^eq, and the Maxwell-Juttner closed-form moments.
"""
from .core import (Lattice, OracleRLB, build, equilibrium_appendix_cell, equilibrium_cell, landau_cell, lattice_path,
                   moments_cell, read_lattice, tau_prime)

__all__ = ["Lattice", "OracleRLB", "build", "equilibrium_appendix_cell", "equilibrium_cell", "landau_cell", "lattice_path", "moments_cell",
           "read_lattice", "tau_prime"]
