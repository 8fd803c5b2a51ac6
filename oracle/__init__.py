"""FP64 CPU oracle for the polynomial multigrid SIPG Poisson solver (Stiller, arXiv 1612.04796).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library under
``paper_1612_04796_gb300/csrc`` and its Python binding) imports, calls or links
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA path: the only
module both sides use is the seeded input generator
``paper_1612_04796_gb300.inputs``, which holds none of the method's arithmetic.

The oracle is written to be read against the paper, not to be fast:

* ``gll``       Section 2: GLL nodes, weights, Lagrange basis and its derivative.
* ``sipg``      Section 2, Eq. (ip) and Eq. (A): the SIPG matrix assembled with
                3D element and face loops (3D GLL quadrature), the 1D matrices,
                the mass matrix and the weak right-hand side.
* ``schwarz``   Section 3.1: element-centred subdomains, overlap rules, the
                hat-shaped weights, and the additive Schwarz smoother with each
                restricted matrix A_ss inverted directly (no fast diagonalisation).
* ``multigrid`` Section 3.2, Algorithm 1: polynomial levels, embedded
                interpolation, the coarse pseudo-inverse solve, the V-cycle,
                standalone MG and the inexact preconditioned CG.

Graded meshes (element widths varying along each axis, an extension of the
paper's uniform grids) go through the same functions: ``sipg.Mesh(widths=...)``
assembles element by element, and ``schwarz.SchwarzSmoother`` then factors
every subdomain's own A_ss.

Readings of passages the paper leaves silent, ambiguous or garbled are stated in
the docstring of the function that adopts them.

Parity unpinned: the hat-weight transition for N_O >= 2 node layers (the paper
defers the definition of w_H to an earlier reference); see
``schwarz.layer_delta``.
"""
