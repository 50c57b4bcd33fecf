"""Plain FP64 CPU oracle of the doubly-periodic slab spectral Ewald solve.

TEST INFRASTRUCTURE. This package exists only to check the CUDA path. Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run anything in it.
The product (``paper_2101_07088_b300``) never imports it, and it imports
nothing from the product.

It follows the paper (Maxian, Pelaez, Greengard, Donev, "A fast spectral
method for electrostatics in doubly-periodic slit channels") step by step at
the same discretisation the GPU path uses:

* ``params``      Sec. 5.1 and 5.3, Table (ewconstraints): cutoffs, grid, xi.
* ``chebyshev``   the second-kind Chebyshev grid of Sec. 5.1 / 5.2.2 and the
                  Chebyshev interpolant (values <-> coefficients).
* ``kernels``     Eq. (gcharge), (spreadkernelEw), (Gnear), (GnearK), (EnearK).
* ``bvp``         Appendix A: the spectral-integration boundary value solver,
                  written as the dense system Eq. (blocksys).
* ``correction``  Sec. 3.1.2 / 4.3.3: the harmonic correction Eq. (inphisc)
                  (with its denominator re-derived, see that module) and the
                  k=0 mode of Sec. 4.3.4.
* ``solver``      Sec. 5.2.2 steps 1-7 plus the near field, the gauge and
                  the energy/force assembly Eq. (Ufinal), (fqE).
* ``brute``       method-independent reference: direct Fourier sums over the
                  periodic lattice and the full dielectric image series, used
                  only to pin the oracle.

Every function is written for a reader checking it against the paper, not
for speed. Numbers are float64 throughout.
"""
