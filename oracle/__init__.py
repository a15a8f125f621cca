"""FP64 CPU oracle for the Neel-rotation Fokker-Planck hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is a plain, slow, obviously correct restatement of what the method
computes (Section 2.1 of the paper: Eqs. for the mean moment, the
Fokker-Planck equation on the sphere and its drift field, with the Neel
constants; Section 2.2 for the normalised signal phi_hat):

* ``physics``    -- material constants -> p1..p4, tau, sigma, beta; the drift
                    field b(m, H, n); the applied fields (Sections 2, 2.1, 2.4).
* ``sphere``     -- real spherical harmonics and tangential gradients, tensor
                    product quadrature on the sphere.
* ``galerkin``   -- Galerkin matrices of the Fokker-Planck operator obtained
                    by quadrature of the weak form (no closed-form coupling
                    coefficients); Boltzmann initial state.
* ``radau``      -- adaptive Radau IIA (order 5) for dc/dt = A(t) c, with the
                    coefficients derived from the collocation definition.
* ``solve``      -- one instance -> m(t_j), dm/dt(t_j), the voltage channels
                    and phi_hat (Section 2.2, model M1 definition of phi_hat).
* ``equilibrium``-- Langevin function (Section 2.2, M0) and brute-force
                    Boltzmann quadrature, used as pins.
* ``legendre1d`` -- an independent 1-D Legendre Galerkin solver for the
                    axially symmetric special cases, used as a pin.
* ``mlp``        -- float64 reference of the surrogate MLP forward/backward.

Every function cites the passage it follows.  Parity status of each
function is listed in its module header.
"""
