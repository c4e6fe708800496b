"""FP64 CPU oracle for the MLFMA-SMR matrix-vector product (arXiv 2407.21724).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2407_21724_gb300``) never imports it, and
this package never imports the product: the two share no code.  The only module
both sides use is ``paper_2407_21724_gb300.workloads``, which draws seeded
synthetic scenes and holds none of the method's arithmetic.

Everything here is plain NumPy/SciPy in float64/complex128, written to be read
against the paper, not to be fast:

* ``special``  - spherical Bessel/Hankel, Riccati-Bessel, Legendre, real
  spherical harmonics and their surface gradients, Gauss-Legendre rules.
* ``sphere``   - closed-form static modes of a sphere (Sec. III, Eqs. 21-25),
  the closed-form self block Z_s (Eq. 16 with delta=1), surface quadrature.
* ``mie``      - single-sphere Mie series (textbook closed form used as a pin).
* ``pmchwt``   - the Galerkin PMCHWT operator (Eqs. 10-19) by direct double
  quadrature: off-diagonal blocks, right-hand sides, dense matvec, far field,
  cross sections, near field.
* ``mlfma``    - the MLFMA operator step by step (Sec. IV, Eqs. 22-26): tree,
  k-space sampling, patterns, translation function, Lagrange interpolation and
  its weighted adjoint, aggregation, translation, receive, near SpMV.
* ``gmres``    - right-preconditioned GMRES (the iterative solve of Sec. V).
* ``mlp``      - FP64 forward/backward/Adam for the learned initial guess.

Sign conventions (the paper's equations disagree with one another, so one
reading is fixed here and used everywhere):

* time dependence e^{j omega t}; g(R) = exp(-j k R) / (4 pi R)   (Eq. 6);
* T_mn = -j k <<psi_m . G . psi_n>> with the dyadic Green's function
  G = (I + grad grad / k^2) g   (Eq. T_far1 and the dyadic below it), i.e. the
  mixed-potential form  -j k <<psi.psi' g>> + (j/k) <<div psi  div' psi' g>>;
* K_mn = - <<psi_m . (psi_n x grad' g)>>: Eq. 9 with n x n x acting as minus
  the tangential projection on the tangential test function; this is also the
  sign of the k-space form Eq. 25;
* right-hand side [<psi, E_inc>, <psi, H_inc>]   (Eqs. 5, 18, 19);
* with these, the unknowns are J = -n x H and M = -E x n on the outer side
  of each surface, and the scattered field is E_s = -zeta L{J} + K{M}.
"""
