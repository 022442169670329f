"""CPU oracle for the Monte Carlo hot path of Volkov's 5-loop QED method
(arXiv:1905.08007).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (``paper_1905_08007_b300``) never imports, links or runs
anything in here, and nothing in here imports the product.

Every function is a plain, slow restatement of what the paper (or the textbook
definition it relies on) says, in float64 unless stated otherwise:

* ``graphs``    -- diagram enumeration, mirror map, gauge classes (k,m,n),
                   UV degree omega, I-closure and Deg (Sec. 2, Sec. 3, Table 1).
* ``philox``    -- the Philox4x32-10 counter generator (Sec. 3, Calc 2; the
                   generator itself is Salmon et al., SC'11).
* ``pdf``       -- Hepp sectors and the Deg-based density of Eq. (1).
* ``polys``     -- Feynman-parametric graph polynomials (Sec. 2, item 4).
* ``dirac``     -- explicit 4x4 Dirac algebra and the F2(0) projection.
* ``integrand`` -- the per-diagram subtracted integrand (Sec. 2, items 1-4).
* ``estimator`` -- the nonadaptive Monte Carlo estimator and run merging
                   (Sec. 3).

Functions whose result the tests cannot tie to anything outside the oracle say
"parity unpinned" in their docstring.
"""
