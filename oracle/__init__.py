"""FP64 CPU oracle of the LB-SMRT collide-and-stream scheme (Yan & Shan, arXiv 2401.11086).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The product path
(``paper_2401_11086_gb300``) never imports, calls or links anything here, and nothing here
imports the product path: the two share no code, tables or constants.

It is a plain, slow, obviously correct restatement of the paper's method in float64 numpy
(complex128 where a caller asks for complex-step derivatives):

* ``lattice``   velocity sets as Gauss-Hermite quadratures (Sec. 3, Eqs. an/fi; Table 3)
* ``hermite``   Hermite polynomials, multi-index and full-tensor forms (Sec. 2.2, Table 1,
                Appendix B)
* ``tensors``   symmetric products, traces and the irreducible projectors of Appendix A
                (Eq. IrrDecomp, Eq. bd, Table 5), by explicit permutation sums
* ``smrt``      the collision (Eq. SMRT), the binomial transform between frames, the rebuild
                (Eq. fi), streaming with the shifted stencil (Sec. 4.1) and the shock
                boundaries (Sec. 4.2)
* ``shock``     Rankine-Hugoniot states (Eq. rankine), shift choice and relaxation times
                (Tables 3 and 4)
* ``adjoint``   the discrete adjoint of one step with respect to f and the relaxation times

Parity status of every function is stated in its module header.
"""
