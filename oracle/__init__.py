"""Plain FP64 CPU oracle of the coupled lattice-Boltzmann / dynamic-immersed-
boundary time step (BGK collide + stream with Guo forcing, Zou-He faces,
quadratic Bouzidi-Firdaouss-Lallemand walls, moving-least-squares
interpolation/spreading, spring-network membrane, Verlet and Newton-Euler
updates, FP64 capsule diagnostics).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import, call or execute anything in
this package.  The CUDA library never uses it, and it uses nothing of the CUDA
library: the two share only the seeded input generators
(``paper_2207_06043_gb300.geometry`` / ``.meshes``), which carry none of the
method's arithmetic.

Each function follows the passage of the paper it cites, in the paper's order
and notation, with numpy primitives as steps and no fusion or reordering beyond
what the equations state.  Readings taken where the paper is silent or garbled
are marked "Reading" in the docstrings.
"""
from . import lattice, ib, membrane, sim  # noqa: F401
