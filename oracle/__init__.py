"""CPU FP64 oracle for the GSPM micromagnetics time step (arXiv 2510.09812, CuPyMag).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, readable NumPy/SciPy restatement of the
paper's equations, used to check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference leg may import it; the library never does, and it
shares no code with the library (the seeded input generator ``synth`` is the only common module,
and it holds none of the method's arithmetic).

Modules
-------
mesh      periodic wrap (Sec. 2.5), node adjacency, reverse Cuthill-McKee order, element geometry
fem       stiffness / mass / RHS matrices (Eqs. LHS, RHS_F, RHS_b), derivatives, volume average
material  reduced constants, cubic stiffness, spontaneous strain (Table A.1), local fields,
          ellipsoid demagnetising factors (Carlson R_D)
solvers   textbook unpreconditioned conjugate gradients (Sec. 2.5)
gspm      one Gauss-Seidel projection step (Algorithm B.1) with magnetostatics and elasticity,
          the stand-alone elastic solve, and the micromagnetic energy (Eq. 1)

Parity unpinned (internally consistent, but no value printed in the paper pins them): the
Gauss-Seidel ordering of the second row of Algorithm B.1 (the paper's print is not a
Gauss-Seidel sweep; the cited scheme's ordering is used), which fields are held fixed when h is
re-evaluated at m*, the CG initial guesses, and how defects enter the magnetisation unknowns.
"""
