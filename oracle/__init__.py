"""FP64 CPU oracle for the rigidly constrained immersed-boundary Stokes solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never calls it and shares no code with it.

Every function is a plain, slow, direct statement of what the paper defines
(Kallemov, Bhalla, Griffith, Donev, "An Immersed Boundary Method for Rigid
Bodies", arXiv:1505.07865), in float64 NumPy:

* ``peskin``     -- the 4-point Peskin kernel phi (Sec. III.A, kernel of the
                    paper's ref. IBM_PeskinReview).
* ``bkp6``       -- the six-point kernel of Bao, Kaye and Peskin that the
                    paper uses (Sec. III.A, ref. New6ptKernel), solved from
                    its defining moment, even-odd and sum-of-squares
                    conditions; ``Grid(kernel="bkp6")`` selects it for J, S.
* ``mac``        -- staggered (MAC) grid, gradient G, divergence D = -G^T,
                    vector Laplacian, viscous operator A (Sec. III.B, Eq. A_def).
* ``ib``         -- interpolation J, spreading S, S~ = S - vol^-1 1^T,
                    rigid-body map K and K^T, the body rotation Q(q) of a
                    unit quaternion (Sec. III.A, III.D, Sec. II).
* ``system``     -- the constrained saddle-point operator (Eq. constrained_Stokes
                    / constrained_periodic), its right-hand side, and a dense
                    bordered LU solve on tiny grids.
* ``fft_stokes`` -- the exact periodic Stokes solution operator L^-1 by the DFT
                    (Eq. L_inv_periodic) and the exact Schur-complement route
                    M Lambda = -(W + J v~) (Eqs. lambda_sol, mob_def).
* ``mobility``   -- the approximate mobility M~ (Eq. M_tilde_ij): RPY form
                    (Eq. RPYTensor) with the periodic correction of App. A, and
                    the 2-D steady form of App. B (Eq. fg_steady_2d).

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force and an independent route
(dense LU vs DFT): among them the rotation direction of K and Q(q) by
hand-computed rotations, and the whole constrained solve by first-order
convergence to the analytic flow of a spinning disk inside a fixed ring
(``test_oracle_convergence.py``, the 2-D analogue of Sec. VII.C), and the
six-point kernel by its defining conditions, three continuous derivatives
and the hydrodynamic radius a = 1.47 h the paper quotes (Sec. IV.A)
(``test_oracle_bkp6.py``).  ``mobility.mtilde_2d_steady`` evaluates the App. B
functional form with caller-supplied coefficients (the paper does not print
them); the form is pinned by its stated limits, the coefficient values are an
input, not an oracle claim.
"""
