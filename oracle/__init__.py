"""FP64 CPU oracle of the mesh-based registration hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call anything in this package.
The CUDA library never calls it, and it shares no code, table or helper with
the CUDA path: it is written independently from the paper, in plain numpy /
scipy, in float64, one function per step of the method, each citing the
equation or section it follows.

Modules
  bspline   cubic B-spline prefilter (Unser's recursion) and evaluation
  mesh      mesh topology, Eq. 9 / Eq. 10 gradients, Eq. 11-13 umbrella
            operator, P1 mass / stiffness matrices
  register  Algorithm 1 (setup, sampling, force, update / solve, energy),
            dense warp and MSD
  adjoint   the warp-plus-SSD energy of a node displacement and its exact
            gradient with respect to the node displacements

Parity status
  Every function here is pinned by a ``-m "not gpu"`` test against a fact
  that does not come from the oracle itself (closed forms, a dense direct
  solve, brute force, invariants, hand-derived values in tests/golden).  The
  one part that stays "parity unpinned" is the end-to-end trajectory of many
  iterations on a phantom: beyond the closed-form ramp trajectory, the
  invariants and the monotone-energy check, nothing outside the oracle fixes
  those numbers (the paper's own results need its brain-CT data).
"""
