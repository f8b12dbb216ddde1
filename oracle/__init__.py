"""FP64 CPU oracle for the nonlinear FE-HMM / FE^2 method (Eidel, Fischer, Gote).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method in numpy/scipy (float64 throughout).  It
exists to check the CUDA path; only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it.  It shares no code with the
CUDA path: the only common module is `synth`, which produces input data.

Modules
  material  compressible neo-Hookean law (Sec. 6, Eq. NH-free-energy ... Aijkl) and the
            St. Venant-Kirchhoff law (Sec. 6, linear elasticity with geometrical nonlinearity)
  rve       periodic RVE: residual, tangent, Newton, averages, condensation and
            the paper's literal saddle-point stiffness transfer (Sec. 3.2, 3.3); law
            selectable, load continuation
  kubc      RVE with kinematic uniform (Dirichlet) boundary conditions (Sec. 3.2, Sec. 4)
  macro     macro Q1/Hex8 mesh, F at quadrature points, HMM assembly (Sec. 3.1)
  driver    nested (Algorithm 1) and alternating (Algorithm 2) load-step schemes
  mlp       the surrogate network: forward, input gradient and Hessian, Sobolev loss and
            its parameter gradient (no counterpart in the paper)
  surrogate the surrogate energy's chain rule to P and dP/dF and its trust distance

Parity status: every function is pinned by tests under tests/ (closed forms,
finite differences, invariants, the paper's Lame table, brute force); none is
"parity unpinned".
"""
