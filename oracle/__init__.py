"""FP64 CPU oracle for Nievergelt's parallel-in-time method (Barker, arXiv 1304.6514).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library: its inputs come from ``workloads`` (random draws and sizes only)
and everything it computes is written here, slowly and plainly, in float64.

Modules
  nievergelt   slice grid, fine schemes, right-hand sides, map fits (PL,
               bilinear, affine), composition, serial fine solve, affine scan,
               FP64 residual refinement
  chebyshev    backward Euler + Lagrange interpolation on Chebyshev-Lobatto
               nodes, the configuration of the paper's Table 1
  mlp          FP64 forward/backward of the slice-conditioned MLP propagator
  wave         Chebyshev spectral wave equation with leapfrog steps on the
               doubled state (Section 5), its affine maps and serial solve

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, a paper value or brute force, except where its docstring says
"parity unpinned".
"""
