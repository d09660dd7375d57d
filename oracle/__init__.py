"""FP64 CPU oracle for the H(div)-DG Darcy/Brinkman multigrid (test infrastructure).

This package is test infrastructure only: it is the plain, slow, obviously
correct statement of what the GPU path computes, used by the tests, by the
smoke check and by the CPU-baseline leg of the benchmark.  The product path
never imports it.  It shares no code with the CUDA library.

Contents (each function cites the passage of Kanschat, Lazarov & Mao,
"Geometric multigrid for Darcy and Brinkman models of flows in highly
heterogeneous porous media", arXiv:1602.04858, that it follows):

* ``basis``      1-D Gauss / Gauss-Lobatto nodes and Lagrange polynomials
                 (nodal tensor basis of RT_k x Q_k, Sec. 2.3).
* ``fem``        global dof layout, assembly of the interior-penalty form
                 a_h (eq. ipbrinkman) and the saddle-point form A_h
                 (eq. Brinkman-weak), right-hand sides (eq. BCh).
* ``multigrid``  nested levels, injection I_j and its transpose (Sec. 3.1,
                 eq. 3), vertex patches, Ritz projections and the symmetric
                 multiplicative Schwarz smoother (Sec. 3.3, eq.
                 smoother-Multiplicative), the (variable) V-cycle (Sec. 3.2).
* ``krylov``     right-preconditioned flexible GMRES (Sec. 3.2, Sec. 4.1).
* ``cnn``        FP64 reference of the learned-initial-guess network (not in
                 the paper): 3x3 convolutions, ReLU, mean squared error and
                 their gradients, in plain loops and NumPy.

Parity unpinned: the GMRES iteration counts of the paper's Tables 1-4 (their
permeability fields are not available), only their trend is checked.
"""
