"""Plain, slow FP64 CPU oracle for deflated BiCGStab on Wilson-Dirac systems.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: it is used by the tests, by the smoke check and by the benchmark's
CPU-baseline leg, and by nothing else.  It shares no code with the CUDA
library (no kernels, headers, tables or helpers); the only thing both sides
share is the seeded input generator in ``inputs/``.

Every routine is written for a reader checking it against the paper
(Abdel-Rehim, Morgan, Wilcox, "Deflated BiCGStab for linear equations in QCD
problems", Lattice 2007) and against the published methods it cites:

  dirac.py    Wilson-Dirac operator A = 1 - kappa*D (+ i*mu*gamma5), Sec. 1
              and Sec. 4; gamma5-hermiticity, Sec. 1.
  kappa.py    kappa_c from the rightmost eigenvalue of D, Sec. 3.
  krylov.py   BiCGStab (van der Vorst 1992), GMRES-DR(m,k) (Morgan 2002,
              cited in Sec. 1), the left-right projection of Sec. 2
              (D-BiCGStab(k)), and the minimal-residual projection over
              previous solutions of Sec. 4.
  evenodd.py  even-odd (Schur) preconditioned operator, Sec. 3 and Sec. 4.
  grad.py     gradients of L = Re(eta^dagger A^{-1} b) (not in the paper).

All arithmetic is complex128 / float64 with numpy; library primitives
(matmul, lstsq, eig, qr, solve) are used only as whole steps.
"""
