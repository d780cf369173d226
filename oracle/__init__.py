"""Plain, slow CPU oracle for the quasi-Monte Carlo evaluation of sector-decomposed Feynman integrals.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or execute anything in this
package; only the test-suite, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
code with the GPU path: the two meet only through the integral definitions and seeded inputs of the
`workloads` module.

What it computes, following Li, Wang, Yan, Zhao, "Efficient Numerical Evaluation of Feynman Integrals"
(Chin. Phys. C 40 (2016) 033103):

  feynman.py    U and F from the momentum representation (Sec. II, Eq. 2), exact rational arithmetic;
                 plus the spanning-tree / 2-forest construction from the graph (cited in Sec. II)
  sectors.py    primary sectors (Eqs. 3-6), iterated decomposition until U and F factorise (Eqs. 7-9),
                 the exponents alpha + beta*eps of Eq. (9); the geometric decomposition the paper prefers
                 (normal fan of the Newton polytope, Sec. II after Eq. 9); Hepp sectors as a third strategy
  prefactor.py  Gamma(N_nu - L D/2)/prod Gamma(nu_j) as a truncated Laurent series in eps (Eq. 2)
  lattice.py    primes, the rank-1 lattice rule (Eq. 17), random shifts (Eqs. 18-20), a plain CBC search
  qmc_oracle.c  the per-point sector integrand: periodising transform (Eq. 21), contour deformation (Eq. 14)
                 with its Jacobian, endpoint subtraction (Eqs. 10-12), eps expansion; and plain lattice sums
  integrate.py  sector sums -> per-shift estimates Q_k -> mean and error (Eqs. 16, 18-20)
  taylor.py     Eq. (11) for endpoint exponents alpha <= -1 of any order (undeformed sectors, numpy, slow):
                 the groundwork for squared propagators, which the GPU path does not take yet

Pins (tests/test_oracle_*.py): textbook U/F forms and the graph construction; closed forms of the massless
and massive bubble, the massive triangle and the massless box; direct simplex cubature of the undecomposed
integrand; the unexpanded subtracted integrand's Laurent coefficients by contour integration in eps;
exactness of the lattice rule on trigonometric polynomials; brute-force CBC; error-estimator coverage;
independence of the total from the decomposition strategy and from lambda; the geometric cones tiling the
space of log x; the paper's printed Laurent coefficients of Tables 2 and 3 (tests/golden/); and, for taylor.py,
the closed forms of massless bubbles with raised powers (alpha = -2, -3) at every order, the C oracle on
alpha = -1 sectors, and strategy independence of the massless box with a squared propagator.
"""
